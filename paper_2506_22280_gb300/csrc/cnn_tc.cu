// The weight-predictor CNN on the tensor cores: forward (training and inference) and parameter gradient
// with BF16 operands and FP32 accumulation in tensor memory (tcgen05, sm_103a).
//
// Activations live in BF16, NHWC, exactly as the GEMMs consume them: the post-ReLU output of every
// convolution is rounded once by the epilogue that produces it (the rounding the tensor cores would
// apply anyway), its sign is the ReLU mask of the backward.  Every GEMM is one launch of one kernel
// template: 128 threads per CTA, looping over 128-row tiles of C; the four warps fill a ring of 2-4 stages of 64-deep K slices of
// A and B with 16-byte cp.async copies (zero-filled where an operand is padding), one thread issues the
// four 128 x BN x 16 MMAs of a slice and commits them to the slice's mbarrier, and the accumulator goes
// through a per-role epilogue.  Operands are read in place, K-major or MN-major:
//   forward conv        C[pixel][co] = im2col(act)[pixel][(tap, ci)] W[co][(tap, ci)]^T   (A gathered)
//   data gradient       one GEMM per output-pixel parity class (py, px) of the stride-2 convolution:
//                       the input pixel (2Y + py, 2X + px) receives only the taps with ky = 1 (py = 0) or
//                       ky in {0, 2} (py = 1), and likewise in x, so
//                       dX_class[(b, Y, X)][ci] = sum over the class's taps and co of
//                       dY[(b, y(Y, ky), x(X, kx))][co] W[co][ky][kx][ci] -- no col2im
//   weight gradient     dW[(tap, ci)][co] = sum over pixels of im2col(act)[pixel][(tap, ci)] dY[pixel][co],
//                       both operands MN-major (channel-contiguous), split over pixels
//   dense layer         feat W1^T (split K), its weight and data gradients with MN-major operands.
// Epilogues fuse what surrounds each GEMM: bias and ReLU with the BF16 rounding (forward), the ReLU mask
// of the layer below with the BF16 rounding of its gradient and per-CTA column sums for its bias
// gradient (data gradient), transposed partial stores (weight gradients).  The first convolution has a
// single input channel (K = 9) and runs on the SIMT pipes with the same rounded operands.
// Every mbarrier wait is bounded; a K-loop wait that gives up sets *status and the CTA drains its own
// MMAs (default bound) before it frees its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "digs_internal.h"
#include "tcgen05.cuh"

namespace digs {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kThr = 128;
constexpr int kBM = 128, kBK = 64;

// ---- geometry of the network (cnn.cu holds the parameter layout) --------------------------------
constexpr int kCh[5] = {1, 32, 64, 128, 128};
constexpr int kEdge[5] = {128, 64, 32, 16, 8};
constexpr int kFeat = 8192, kFeatPitch = 8200, kHid = 128;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void unpack8(const uint4& u, float f[8]) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}

// 16-byte asynchronous copy global -> shared; src == nullptr fills the 16 bytes with zeros (no bytes read).
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, const void* valid_any) {
  const int n = src ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src ? src : valid_any), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- operand loaders -------------------------------------------------------------------------------
// K-major loaders return the address of the 8 reduction elements [k, k + 8) of operand row `row`;
// MN-major loaders the address of the 8 row elements [mn, mn + 8) at reduction index k; nullptr where
// the operand is zero.  kdim(K) is the reduction length of the CTA's GEMM.

struct PlainK {  // X[row][k] = p[row * ld + k]
  const bf16* p;
  int ld, rows;
  __device__ const bf16* kchunk(int row, int k) const { return row < rows ? p + (size_t)row * ld + k : nullptr; }
  __device__ int kdim(int K) const { return K; }
  __device__ int zsplit() const { return blockIdx.z; }
};

struct PlainMN {  // X[mn][k] = p[k * ld + mn]
  const bf16* p;
  int ld, cols;
  __device__ const bf16* mnchunk(int mn, int k) const { return mn < cols ? p + (size_t)k * ld + mn : nullptr; }
  __device__ int kdim(int K) const { return K; }
  __device__ int zsplit() const { return blockIdx.z; }
};

// Implicit im2col of a 3 x 3, stride-2, padding-1 convolution over an NHWC input H x W x C (powers of
// two, C >= 8): row p = output pixel (b, y, x), column (tap, c) = in[b][2y + ky - 1][2x + kx - 1][c].
struct ConvGeomB {
  const bf16* act;
  int H, lwo, lc, rows, cols;  // input height (= width); log2 output width; log2 C; pixels; 9 C
  __device__ const bf16* at(int p, int kk) const {
    if (p >= rows || kk >= cols) return nullptr;
    const int tap = kk >> lc, c = kk & ((1 << lc) - 1), ky = tap / 3, kx = tap - 3 * ky;
    const int x = p & ((1 << lwo) - 1), y = (p >> lwo) & ((1 << lwo) - 1), b = p >> (2 * lwo);
    const int iy = 2 * y + ky - 1, ix = 2 * x + kx - 1;
    if (iy < 0 || iy >= H || ix < 0 || ix >= H) return nullptr;
    return act + ((((size_t)b * H + iy) * H + ix) << lc) + c;
  }
};
struct ConvK {  // A = im2col, rows = output pixels, reduction = (tap, c)
  ConvGeomB g;
  __device__ const bf16* kchunk(int row, int k) const { return g.at(row, k); }
  __device__ int kdim(int K) const { return K; }
  __device__ int zsplit() const { return blockIdx.z; }
};
struct ConvMN {  // A = im2col^T, rows = (tap, c), reduction = output pixels
  ConvGeomB g;
  __device__ const bf16* mnchunk(int mn, int k) const { return g.at(k, mn); }
  __device__ int kdim(int K) const { return K; }
  __device__ int zsplit() const { return blockIdx.z; }
};

// Taps (ky, kx) that reach input pixels of parity class z = 2 py + px, and the offset of the class's
// weight block (in units of N C) in the class-ordered transposed weights.
__device__ __forceinline__ int class_taps(int z) { return (z == 0) ? 1 : (z == 3 ? 4 : 2); }
__device__ __forceinline__ int class_off(int z) { return z == 0 ? 0 : (z == 1 ? 1 : (z == 2 ? 3 : 5)); }
__host__ __device__ __forceinline__ void class_tap(int z, int t, int& ky, int& kx) {
  const int py = z >> 1, px = z & 1;
  const int nx = px ? 2 : 1;
  const int ty = t / nx, tx = t - ty * nx;
  ky = py ? 2 * ty : 1;
  kx = px ? 2 * tx : 1;
}

// A of the data-gradient GEMM of class z = blockIdx.z: row (b, Y, X) of the class grid (Ho x Ho, the
// output size of the convolution), reduction (t, co) over the class's taps and the N output channels:
// dY[b][y][x][co] with 2y + ky - 1 = 2Y + py, 2x + kx - 1 = 2X + px.
struct ParityK {
  const bf16* dy;
  int lho, ln, rows;  // log2 Ho; log2 N; rows = B Ho Ho
  __device__ const bf16* kchunk(int row, int k) const {
    if (row >= rows) return nullptr;
    const int z = blockIdx.z, t = k >> ln, co = k & ((1 << ln) - 1);
    int ky, kx;
    class_tap(z, t, ky, kx);
    const int Ho = 1 << lho;
    const int X = row & (Ho - 1), Y = (row >> lho) & (Ho - 1), b = row >> (2 * lho);
    const int y = (2 * Y + (z >> 1) + 1 - ky) >> 1, x = (2 * X + (z & 1) + 1 - kx) >> 1;
    if (y >= Ho || x >= Ho) return nullptr;
    return dy + ((((((size_t)b << lho) + y) << lho) + x) << ln) + co;
  }
  __device__ int kdim(int) const { return class_taps(blockIdx.z) << ln; }
  __device__ int zsplit() const { return 0; }  // blockIdx.z is the class, not a split
};

// B of the data-gradient GEMM: the class's weights transposed, wt[class block][ci][(t, co)].
struct ClassWt {
  const bf16* wt;
  int ln, C;  // log2 N (output channels of the convolution), C input channels (rows)
  __device__ const bf16* kchunk(int row, int k) const {
    if (row >= C) return nullptr;
    const int z = blockIdx.z, kc = class_taps(z) << ln;
    return wt + ((size_t)class_off(z) << ln) * C + (size_t)row * kc + k;
  }
  __device__ int kdim(int K) const { return K; }
};

// ---- epilogues ---------------------------------------------------------------------------------------
// apply(row, col0, v[16], acc): the accumulator's row `row`, columns [col0, col0 + 16) of the CTA's tile
// (global indices); acc is a per-thread running value; finish(...) runs once per thread after all
// columns, with the CTA's shared scratch (all threads call it).

// BF16 rows (+ bias, ReLU): out[(row / group) * gpitch + (row % group) * rpitch + col].
struct EpiBf16 {
  bf16* out;
  const float* bias;
  int relu, rows, group, gpitch, rpitch;
  __device__ void apply(int row, int col0, float v[16], float&, float*) const {
    if (row >= rows) return;
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float a = v[2 * j] + bias[col0 + 2 * j], b = v[2 * j + 1] + bias[col0 + 2 * j + 1];
      if (relu) {
        a = fmaxf(a, 0.f);
        b = fmaxf(b, 0.f);
      }
      w[j] = pack2(a, b);
    }
    uint4* d = reinterpret_cast<uint4*>(out + (size_t)(row / group) * gpitch + (size_t)(row % group) * rpitch + col0);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
  __device__ void finish(int, float, float*, int, int, int) const {}
};

// FP32 rows of split z: part[z * zstride + row * ld + col].
struct EpiF32 {
  float* part;
  long long zstride;
  int rows, ld;
  __device__ void apply(int row, int col0, float v[16], float&, float*) const {
    if (row >= rows) return;
    float4* d = reinterpret_cast<float4*>(part + blockIdx.z * zstride + (size_t)row * ld + col0);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
  __device__ void finish(int, float, float*, int, int, int) const {}
};

// Transposed FP32 store of split z: out[z * zstride + col * ld + row] for row < rows (coalesced: the
// lanes of a warp hold consecutive rows).
struct EpiF32T {
  float* out;
  long long zstride;
  int rows, ld;
  __device__ void apply(int row, int col0, float v[16], float&, float*) const {
    if (row >= rows) return;
    float* d = out + blockIdx.z * zstride + (size_t)col0 * ld + row;
#pragma unroll
    for (int j = 0; j < 16; ++j) d[(size_t)j * ld] = v[j];
  }
  __device__ void finish(int, float, float*, int, int, int) const {}
};

// Sum 16 per-lane values over the warp's 32 lanes by recursive halving (16 shuffles); lane l ends with
// the total of value 8 b4 + 4 b3 + 2 b2 + b1 (b_i = bit i of l).
__device__ __forceinline__ float warp_sum16(float v[16], int lane) {
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool hi = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? v[i] : v[i + half], keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
__device__ __forceinline__ int sum16_col(int lane) {
  return 8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
}

// Data gradient of class z: row (b, Y, X) is input pixel (b, 2Y + py, 2X + px) of a layer with C = BN
// channels and H x H pixels; dY_in = dX * [act > 0] (act: that layer's post-ReLU output), stored in BF16
// at the NHWC index; the masked FP32 values are summed per column over the CTA's rows into
// colpart[z * n_mt + mt][col] (bias gradient of that layer; mt the row tile).
template <int BN>
struct EpiDx {
  bf16* dy_out;
  const bf16* act;
  float* colpart;
  int lho, H, rows;
  __device__ void apply(int row, int col0, float v[16], float&, float* scratch) const {
    const int z = blockIdx.z;
    if (row < rows) {
      const int Ho = 1 << lho;
      const int X = row & (Ho - 1), Y = (row >> lho) & (Ho - 1), b = row >> (2 * lho);
      const size_t idx = (((size_t)b * H + 2 * Y + (z >> 1)) * H + 2 * X + (z & 1)) * BN + col0;
      const uint4* a = reinterpret_cast<const uint4*>(act + idx);
      float m[16];
      unpack8(a[0], m);
      unpack8(a[1], m + 8);
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = m[j] > 0.f ? v[j] : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = pack2(v[2 * j], v[2 * j + 1]);
      uint4* d = reinterpret_cast<uint4*>(dy_out + idx);
      d[0] = make_uint4(w[0], w[1], w[2], w[3]);
      d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
    }
    // column sums over the warp's 32 rows, into the shared scratch [warp][BN] (written in finish order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float s = warp_sum16(v, lane);
    if ((lane & 1) == 0) scratch[warp * BN + col0 - blockIdx.y * BN + sum16_col(lane)] = s;
  }
  __device__ void finish(int, float, float* scratch, int tid, int mt, int n_mt) const {
    __syncthreads();
    if (tid < BN) {
      const float s = scratch[tid] + scratch[BN + tid] + scratch[2 * BN + tid] + scratch[3 * BN + tid];
      colpart[((size_t)blockIdx.z * n_mt + mt) * BN + tid] = s;
    }
  }
};

// Gradient of the dense layer's input, rows b (batch entry) and columns f (feature, blockIdx.y selects
// 128 of them, i.e. one pixel's 128 channels of the last convolution):
// dY3[b][f] = dfeat[b][f] [act3[b][f] > 0] in BF16 (feat holds act3 in its first 8192 columns; the two
// angle inputs get no gradient), and the masked FP32 values summed per column over the CTA's rows into
// colpart[blockIdx.y * n_mt + mt][c] (the last convolution's bias gradient sums those rows).
struct EpiDfeat {
  bf16* dy3;
  const bf16* feat;  // [B][kFeatPitch]
  float* colpart;
  int nb;
  __device__ void apply(int row, int col0, float v[16], float&, float* scratch) const {
    if (row < nb) {
      const uint4* a = reinterpret_cast<const uint4*>(feat + (size_t)row * kFeatPitch + col0);
      float m[16];
      unpack8(a[0], m);
      unpack8(a[1], m + 8);
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = m[j] > 0.f ? v[j] : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = pack2(v[2 * j], v[2 * j + 1]);
      uint4* d = reinterpret_cast<uint4*>(dy3 + (size_t)row * kFeat + col0);
      d[0] = make_uint4(w[0], w[1], w[2], w[3]);
      d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float s = warp_sum16(v, lane);
    if ((lane & 1) == 0) scratch[warp * 128 + col0 - blockIdx.y * 128 + sum16_col(lane)] = s;
  }
  __device__ void finish(int, float, float* scratch, int tid, int mt, int n_mt) const {
    __syncthreads();
    if (tid < 128) {
      const float s = scratch[tid] + scratch[128 + tid] + scratch[256 + tid] + scratch[384 + tid];
      colpart[((size_t)blockIdx.y * n_mt + mt) * 128 + tid] = s;
    }
  }
};

// ---- the GEMM kernel -------------------------------------------------------------------------------
// S stages of (A, B) slices: 4 for long reductions, fewer where a CTA has only a few slices, so that
// more CTAs share an SM (at most five: 5 x 32 ... 2 x 128 tensor-memory columns stay within the 512).
template <int BN, int S>
struct Cfg {
  static constexpr int kA = kBM * kBK * 2;  // bytes of one A slice (16 KB)
  static constexpr int kB = BN * kBK * 2;
  static constexpr int kStage = kA + kB;
  static constexpr int kScratch = 4 * BN * 4;  // epilogue column sums [warp][BN]
  static constexpr size_t kSmem = 1024 + (size_t)S * kStage + 128 + kScratch;
};

// Shared-memory byte offset of a 16-byte chunk: K-major (row, kc) of a ROWS x 64 slice; MN-major
// (mn chunk mc, k) of an MN x 64 slice.
__device__ __forceinline__ uint32_t off_k(int row, int kc) { return (uint32_t)(((row >> 3) * 8 + kc) * 128 + (row & 7) * 16); }
template <int MN>
__device__ __forceinline__ uint32_t off_mn(int mc, int k) {
  return (uint32_t)(((k >> 3) * (MN / 8) + mc) * 128 + (k & 7) * 16);
}

// Fills one operand slice: ROWS (MN extent) x 64 reduction elements starting at (r0, k0); the thread's
// chunks are q = tid + 128 i, laid out so that a warp's copies fill whole 128-byte core-matrix rows.
template <int ROWS, bool MN, class L>
__device__ __forceinline__ void fill(const L& ld, uint32_t sdst, int r0, int k0, int kend, const void* any) {
#pragma unroll
  for (int i = 0; i < ROWS / 16; ++i) {
    const int q = threadIdx.x + kThr * i;
    if constexpr (!MN) {
      const int row = (q & 7) | ((q >> 6) << 3), kc = (q >> 3) & 7;
      const int k = k0 + kc * 8;
      cp16(sdst + off_k(row, kc), k < kend ? ld.kchunk(r0 + row, k) : nullptr, any);
    } else {
      constexpr int G = ROWS / 8;
      const int rest = q >> 3, mc = rest & (G - 1), k = ((rest / G) << 3) | (q & 7);
      cp16(sdst + off_mn<ROWS>(mc, k), k0 + k < kend ? ld.mnchunk(r0 + mc * 8, k0 + k) : nullptr, any);
    }
  }
}

template <int ROWS, bool MN>
__device__ __forceinline__ uint64_t slice_desc(uint32_t a, int j) {
  if constexpr (!MN) return tc::smem_desc(a + j * 256, 128, 1024);
  return tc::smem_desc(a + j * 2 * (ROWS / 8) * 128, (ROWS / 8) * 128, 128);
}

// C tiles (128 x BN) of rows [mt 128, mt 128 + 128) for mt = blockIdx.x, blockIdx.x + gridDim.x, ...
// (n_mt row tiles in all), columns from blockIdx.y BN; blockIdx.z = split of the reduction (kchunk
// each) or, for the data gradient, the parity class (its loaders read blockIdx.z).  The tensor memory
// and the mbarrier ring stay with the CTA across its tiles; g counts the slices issued so far, which
// selects the stage buffer (g mod S) and the mbarrier phase (g div S).
template <int BN, int kStages, bool AMN, bool BMN, class LA, class LB, class EP>
__global__ void __launch_bounds__(kThr, BN == 32 ? 5 : (BN == 64 ? (kStages == 2 ? 4 : (kStages == 3 ? 3 : 2)) : 1)) k_cnn_gemm(const LA la, const LB lb, const EP ep, int n_mt, int K, int kchunk,
                                                      int* status, unsigned wait_limit, const void* any) {
  using C = Cfg<BN, kStages>;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = (uint64_t*)(sm + kStages * C::kStage);
  uint32_t* tslot = (uint32_t*)(bar + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.y * BN;
  const int Kz = la.kdim(K);
  const long long kb0 = (long long)la.zsplit() * kchunk;
  const int kb = kb0 >= Kz ? Kz : (int)kb0;
  const int ke = (int)min((long long)Kz, (long long)kb + kchunk);
  const int nk = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < kStages; ++s) tc::mbar_init(bar + s, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(tslot, BN);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t sbase = tc::smem_u32(sm);
  constexpr uint32_t idesc = tc::idesc_bf16(kBM, BN, AMN, BMN);
  float* scratch = reinterpret_cast<float*>((uint8_t*)bar + 128);  // the epilogue's column sums
  int ok = 1;
  unsigned g = 0;
  // the first S - 1 slices of a tile, into the stage buffers g, g + 1, ... (all free: no MMA in flight)
  auto prologue = [&](int m0) {
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
      if (s < nk) {
        const uint32_t sa = sbase + ((g + s) % kStages) * C::kStage;
        fill<kBM, AMN>(la, sa, m0, kb + s * kBK, ke, any);
        fill<BN, BMN>(lb, sa + C::kA, n0, kb + s * kBK, ke, any);
      }
      cp_commit();
    }
  };
  int mt = blockIdx.x;
  if (mt < n_mt) prologue(mt * kBM);
  while (mt < n_mt) {
    const int m0 = mt * kBM;
    int issued = 0;
    for (int c = 0; c < nk; ++c) {
      cp_wait<kStages - 2>();     // this thread's copies of slice c have landed
      tc::fence_async_smem();     // ... and are visible to the tensor core
      ok = __syncthreads_and(ok);
      if (!ok) break;
      const unsigned gc = g + c;
      if (tid == 0) {
        tc::fence_after();
        const uint32_t sa = sbase + (gc % kStages) * C::kStage, sb = sa + C::kA;
#pragma unroll
        for (int j = 0; j < kBK / 16; ++j)
          tc::mma_bf16(tmem, slice_desc<kBM, AMN>(sa, j), slice_desc<BN, BMN>(sb, j), idesc, (c > 0 || j > 0) ? 1u : 0u);
        tc::mma_commit(bar + gc % kStages);
      }
      issued = c + 1;
      const int nxt = c + kStages - 1;  // refills the buffer of slice c - 1 once its MMAs are done
      if (nxt < nk) {
        if (c >= 1) ok = ok && tc::mbar_wait(bar + (gc - 1) % kStages, ((gc - 1) / kStages) & 1u, wait_limit);
        if (ok) {
          const uint32_t sa = sbase + ((g + nxt) % kStages) * C::kStage;
          fill<kBM, AMN>(la, sa, m0, kb + nxt * kBK, ke, any);
          fill<BN, BMN>(lb, sa + C::kA, n0, kb + nxt * kBK, ke, any);
        }
      }
      cp_commit();
    }
    cp_wait<0>();
    const unsigned gl = g + issued - 1;  // the last slice: its commit tracks all the tile's MMAs
    const bool drained = issued == 0 || tc::mbar_wait(bar + gl % kStages, (gl / kStages) & 1u, tc::kWaitLimit);
    ok = __syncthreads_and(ok && drained);
    tc::fence_after();
    g += issued;
    if (!ok) break;
    // the next tile's first copies go out now, so that they land while this tile's epilogue runs
    const int next = mt + gridDim.x;
    if (next < n_mt) prologue(next * kBM);
    float acc = 0.f;
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (issued == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      ep.apply(row, n0 + c0, v, acc, scratch);
    }
    ep.finish(row, acc, scratch, tid, mt, n_mt);
    // the accumulator and the scratch are free again before the next tile's MMAs
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    mt = next;
  }
  cp_wait<0>();
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, BN);
  }
  if (!ok && tid == 0 && status) atomicExch(status, 1);
}

// ---- SIMT kernels and small steps --------------------------------------------------------------------

// First convolution (1 -> 32 channels, 128^2 -> 64^2): act0[p][co] = relu(b[co] + sum over taps of
// r(w[co][tap]) r(img(tap))), r = BF16 rounding, img the FP32 input; one thread per output pixel, 32
// channels stored as four 16-byte BF16 chunks; the rounded input is also stored (imgb) for the backward.
__global__ void __launch_bounds__(256) k_conv0_fwd(const float* __restrict__ img, const float* __restrict__ w,
                                                   const float* __restrict__ bias, int npix, bf16* __restrict__ out,
                                                   bf16* __restrict__ imgb) {
  __shared__ float sw[32 * 9], sb[32];
  for (int i = threadIdx.x; i < 32 * 9; i += blockDim.x) sw[i] = bf16r(w[i]);
  if (threadIdx.x < 32) sb[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const int x = p & 63, y = (p >> 6) & 63, b = p >> 12;
  float xin[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int iy = 2 * y + t / 3 - 1, ix = 2 * x + t % 3 - 1;
    xin[t] = (iy >= 0 && iy < 128 && ix >= 0 && ix < 128) ? bf16r(img[((size_t)b * 128 + iy) * 128 + ix]) : 0.f;
  }
  // the BF16 input the weight gradient reads: this pixel writes input pixels (2y + dy, 2x + dx), dy, dx in
  // {0, 1} (its taps 4, 5, 7, 8), so every input pixel is written exactly once
  {
    uint32_t* row0 = reinterpret_cast<uint32_t*>(imgb + ((size_t)b * 128 + 2 * y) * 128 + 2 * x);
    row0[0] = pack2(xin[4], xin[5]);
    row0[64] = pack2(xin[7], xin[8]);  // the next row: 128 BF16 = 64 words further
  }
  uint4* d = reinterpret_cast<uint4*>(out + (size_t)p * 32);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int co = 8 * q + j;
      float a = sb[co];
#pragma unroll
      for (int t = 0; t < 9; ++t) a = fmaf(sw[co * 9 + t], xin[t], a);
      o[j] = fmaxf(a, 0.f);
    }
    d[q] = make_uint4(pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]), pack2(o[6], o[7]));
  }
}

// Weight gradient of the first convolution: part[block][co * 9 + tap] = sum over the block's pixels of
// dY0[p][co] img(tap) (both BF16).  Thread t owns the channels 4 (t & 7) ... + 3 and the pixel stream
// t >> 3 (32 streams per block, grid-stride over the pixels, four pixels per step with all their loads
// issued first); its 36 products per pixel accumulate in registers, and the block's 32 streams are
// added in a fixed order through shared memory.
__global__ void __launch_bounds__(256, 4) k_conv0_dw(const bf16* __restrict__ dy, const bf16* __restrict__ img,
                                                     int npix, float* __restrict__ part) {
  __shared__ float red[32][289];
  const int cg = threadIdx.x & 7, sid = threadIdx.x >> 3;
  float acc[4][9];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[j][t] = 0.f;
  const long long stride = (long long)gridDim.x * 32;
#pragma unroll 2
  for (long long p = (long long)blockIdx.x * 32 + sid; p < npix; p += stride) {
    const uint2 u = *reinterpret_cast<const uint2*>(dy + p * 32 + cg * 4);
    const int x = (int)(p & 63), y = (int)((p >> 6) & 63), b = (int)(p >> 12);
    float xv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int iy = 2 * y + t / 3 - 1, ix = 2 * x + t % 3 - 1;
      xv[t] = (iy >= 0 && iy < 128 && ix >= 0 && ix < 128) ? __bfloat162float(img[((size_t)b * 128 + iy) * 128 + ix])
                                                          : 0.f;
    }
    const float d[4] = {__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                        __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u)};
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int t = 0; t < 9; ++t) acc[j][t] = fmaf(d[j], xv[t], acc[j][t]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int t = 0; t < 9; ++t) red[sid][(cg * 4 + j) * 9 + t] = acc[j][t];
  __syncthreads();
  for (int o = threadIdx.x; o < 288; o += blockDim.x) {
    float sum = 0.f;
    for (int k = 0; k < 32; ++k) sum += red[k][o];
    part[(size_t)blockIdx.x * 288 + o] = sum;
  }
}

// out[c] = sum over the rows r < R of in[r * ld + c], in one launch: block (x, y) sums rows
// [y chunk, (y + 1) chunk) of the columns 32 x .. 32 x + 31 (strided over its 8 warps, then the warp sums
// in order) into part[y * cols + c]; the last block of column group x to finish (a ticket counter per
// group, reset by that block) then adds the gridDim.y partials in chunk order.  The result does not depend
// on which block finishes last, and no block waits for another.
__global__ void __launch_bounds__(256) k_colreduce_once(const float* __restrict__ in, int R, int cols, int ld,
                                                        int chunk, float* part, float* __restrict__ out,
                                                        unsigned* tickets) {
  __shared__ float red[8][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int r0 = blockIdx.y * chunk, r1 = min(R, r0 + chunk);
  float s = 0.f;
  if (c < cols)
    for (int r = r0 + warp; r < r1; r += 8) s += in[(size_t)r * ld + c];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && c < cols) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    part[(size_t)blockIdx.y * cols + c] = t;
  }
  __threadfence();  // this block's partials are visible before its ticket is taken
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&tickets[blockIdx.x], 1u) == gridDim.y - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  s = 0.f;
  if (c < cols)
    for (int y = warp; y < (int)gridDim.y; y += 8) s += __ldcg(&part[(size_t)y * cols + c]);
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && c < cols) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    out[c] = t;
  }
  if (threadIdx.x == 0) tickets[blockIdx.x] = 0u;
}

// out[i] = sum over z of part[z * n + i] (+ bias[i % nb] and ReLU when bias != nullptr), in a fixed order:
// 32 outputs per block, warp w adding the splits z = w, w + 8, ... in order (coalesced over the outputs),
// then the eight warp sums added in warp order.
__global__ void __launch_bounds__(256) k_sum_z(const float* __restrict__ part, int Z, long long n,
                                               const float* __restrict__ bias, int nb, float* __restrict__ out) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < n)
    for (int z = warp; z < Z; z += 8) s += part[(size_t)z * n + i];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < n) {
    float t = red[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += red[w][lane];
    if (bias) t = fmaxf(t + bias[i % nb], 0.f);
    out[i] = t;
  }
}

// All of a forward's weight conversions to BF16 in one launch: job k covers the elements [start[k], start[k + 1])
// of a grid-stride loop.  Kind 0, rows: out[r][c] = BF16 of in[r][c] for c < b, 0 for b <= c < c_pitch
// (a rows, row pitch c).  Kind 1, the class-ordered transposed weights of a convolution with N = a output
// and C = b input channels: out[class block z][ci][(t, co)] = BF16 of w[co][ky_t][kx_t][ci] for the
// class's taps t.  Kind 2: out[e] = BF16 of in[e].
struct BfJob {
  const float* in;
  bf16* out;
  int kind, a, b, c;
};
struct BfJobs {
  BfJob job[8];
  long long start[9];
  int count;
};
__global__ void __launch_bounds__(256) k_to_bf16_jobs(const __grid_constant__ BfJobs J) {
  const long long total = J.start[J.count];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < J.count && i >= J.start[k + 1]) ++k;
    const BfJob& jb = J.job[k];
    const long long e = i - J.start[k];
    float x;
    if (jb.kind == 0) {
      const int r = (int)(e / jb.c), c = (int)(e - (long long)r * jb.c);
      x = c < jb.b ? jb.in[(size_t)r * jb.b + c] : 0.f;
    } else if (jb.kind == 1) {
      const long long NC = (long long)jb.a * jb.b;
      const int z = e < NC ? 0 : (e < 3 * NC ? 1 : (e < 5 * NC ? 2 : 3));
      const long long local = e - (long long)class_off(z) * NC;
      const int kc = class_taps(z) * jb.a;
      const int ci = (int)(local / kc), rem = (int)(local - (long long)ci * kc), t = rem / jb.a, co = rem - t * jb.a;
      int ky, kx;
      class_tap(z, t, ky, kx);
      x = jb.in[((size_t)co * 9 + ky * 3 + kx) * jb.b + ci];
    } else {
      x = jb.in[e];
    }
    jb.out[e] = __float2bfloat16_rn(x);
  }
}

// The dense layer's two angle inputs and zero padding: feat[b][8192 + j] = BF16 of (cos, sin, 0, ...).
__global__ void k_feat_tail(bf16* __restrict__ feat, const float* __restrict__ cs, int B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * (kFeatPitch - kFeat)) return;
  const int b = i / (kFeatPitch - kFeat), j = i - b * (kFeatPitch - kFeat);
  feat[(size_t)b * kFeatPitch + kFeat + j] = __float2bfloat16_rn(j < 2 ? cs[2 * b + j] : 0.f);
}

unsigned grid_of(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

// One GEMM launch: M rows of C in 128-row tiles, gy column tiles of BN, gz splits (or classes).
template <int BN, int S, bool AMN, bool BMN, class LA, class LB, class EP>
cudaError_t gemm(const LA& la, const LB& lb, const EP& ep, int M, int K, int gy, int gz, int kchunk, const void* any,
                 cudaStream_t st) {
  using C = Cfg<BN, S>;
  auto kern = k_cnn_gemm<BN, S, AMN, BMN, LA, LB, EP>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (M <= 0) return cudaSuccess;
  // row tiles per CTA: enough CTAs for every SM to hold as many as its shared memory allows, several
  // tiles each when there are more
  const int n_mt = (M + kBM - 1) / kBM;
  const long long per_sm = std::max(1, std::min(5, (int)(227 * 1024 / C::kSmem)));
  const long long total = (long long)n_mt * gy * gz, target = 4LL * 152 * per_sm;
  const int per_cta = (int)std::max(1LL, (total + target - 1) / target);
  const int gx = (n_mt + per_cta - 1) / per_cta;
  kern<<<dim3(gx, gy, gz), kThr, C::kSmem, st>>>(la, lb, ep, n_mt, K, kchunk, nullptr, tc::kWaitLimit, any);
  note_launches(1);
  return cudaGetLastError();
}

#define TC_TRY(...)                       \
  do {                                    \
    cudaError_t e__ = (__VA_ARGS__);      \
    if (e__ != cudaSuccess) return e__;   \
  } while (0)

// Splits of a pixel-reduction weight gradient: about two CTAs per SM over the row tiles, at least four
// 64-pixel slices per split, partials within the buffer.
constexpr int kConv0Ctas = 4 * 152;  // k_conv0_dw: four CTAs per SM (its register limit)
constexpr int kColTickets = 64;      // colreduce ticket counters (column groups of 32)

int dw_splits(int tiles, long long pixels, long long part_floats, long long tile_floats) {
  long long z = (2LL * 152 + tiles - 1) / tiles;
  z = std::min(z, std::max(1LL, pixels / 256));
  z = std::min(z, std::max(1LL, part_floats / tile_floats));
  return (int)std::max(1LL, z);
}
int chunk_of(long long n, int z) { return (int)(((n + z - 1) / z + kBK - 1) / kBK * kBK); }

// out[c] = sum over r < R of in[r * ld + c] in a fixed order: row chunks of 64 summed into scratch by
// many blocks, then the chunk sums by one block per 32 columns (one pass when R <= 512).
// tickets: (cols + 31) / 32 counters, zero on entry (and left zero).
cudaError_t colreduce(const float* in, int R, int cols, int ld, float* out, float* scratch, unsigned* tickets,
                      cudaStream_t st) {
  const unsigned gx = (unsigned)((cols + 31) / 32);
  const int chunk = R <= 2048 ? 64 : 128, nch = (R + chunk - 1) / chunk;
  k_colreduce_once<<<dim3(gx, nch), 256, 0, st>>>(in, R, cols, ld, chunk, scratch, out, tickets);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

// ---- host side -------------------------------------------------------------------------------------

size_t cnn_tc_layout(void* base, int B, CnnTc* t) {
  size_t off = 0;
  char* p = (char*)base;
  auto take = [&](size_t bytes) -> void* {
    void* q = p ? p + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return q;
  };
  CnnTc w{};
  w.imgb = (uint16_t*)take((size_t)B * 128 * 128 * 2);
  for (int l = 0; l < 3; ++l) w.act[l] = (uint16_t*)take((size_t)B * kEdge[l + 1] * kEdge[l + 1] * kCh[l + 1] * 2);
  w.feat = (uint16_t*)take((size_t)B * kFeatPitch * 2);
  w.dy[0] = (uint16_t*)take((size_t)B * 4096 * 32 * 2);  // dY of conv 2, then of conv 0
  w.dy[1] = (uint16_t*)take((size_t)B * 1024 * 64 * 2);  // dY of conv 1
  w.dy3 = (uint16_t*)take((size_t)B * kFeat * 2);
  w.dhb = (uint16_t*)take((size_t)B * kHid * 2);
  for (int l = 1; l < 4; ++l) {
    w.wb[l] = (uint16_t*)take((size_t)kCh[l + 1] * 9 * kCh[l] * 2);
    w.wt[l] = (uint16_t*)take((size_t)kCh[l + 1] * 9 * kCh[l] * 2);
  }
  w.wb[0] = w.wt[0] = nullptr;
  w.w1b = (uint16_t*)take((size_t)kHid * kFeatPitch * 2);
  w.part_floats = std::max<long long>(16LL * B * kHid, 5LL << 20);
  w.part = (float*)take((size_t)w.part_floats * 4);
  w.colpart_floats = std::max<long long>({1024LL * B, 8192LL * ((B + 127) / 128), (long long)kConv0Ctas * 288});
  w.colpart = (float*)take((size_t)w.colpart_floats * 4);
  w.tickets = (unsigned*)take(kColTickets * sizeof(unsigned));
  if (t) *t = w;
  return off;
}

cudaError_t cnn_tc_forward(const CnnNet& net, const float* img, const float* cs, int B, const CnnTc& t, float* h,
                           cudaStream_t st) {
  // BF16 copies of the weights, row-major (forward) and class-ordered transposed (data gradient): one
  // launch (the first convolution rounds the input images itself and stores their BF16 copy)
  BfJobs J{};
  long long at = 0;
  auto add = [&](const float* in, bf16* out, int kind, int a, int b, int c, long long n) {
    J.job[J.count] = BfJob{in, out, kind, a, b, c};
    J.start[J.count++] = at;
    at += n;
  };
  for (int l = 1; l < 4; ++l) {
    const int N = kCh[l + 1], Kl = 9 * kCh[l];
    add(net.w[l], (bf16*)t.wb[l], 0, N, Kl, Kl, (long long)N * Kl);
    add(net.w[l], (bf16*)t.wt[l], 1, N, kCh[l], 0, (long long)N * Kl);
  }
  add(net.w1, (bf16*)t.w1b, 0, kHid, kFeat + 2, kFeatPitch, (long long)kHid * kFeatPitch);
  J.start[J.count] = at;
  k_to_bf16_jobs<<<grid_of(at), 256, 0, st>>>(J);
  const int npix0 = B * 4096;
  k_conv0_fwd<<<(npix0 + 255) / 256, 256, 0, st>>>(img, net.w[0], net.b[0], npix0, (bf16*)t.act[0], (bf16*)t.imgb);
  note_launches(2);
  const void* any = t.wb[1];
  for (int l = 1; l < 4; ++l) {
    const int H = kEdge[l], lwo = l == 1 ? 5 : (l == 2 ? 4 : 3), lc = l == 1 ? 5 : (l == 2 ? 6 : 7);
    const int rows = B * kEdge[l + 1] * kEdge[l + 1], N = kCh[l + 1], Kl = 9 * kCh[l];
    const ConvK A{ConvGeomB{(const bf16*)t.act[l - 1], H, lwo, lc, rows, Kl}};
    const PlainK Bw{(const bf16*)t.wb[l], Kl, N};
    if (l == 1) {
      const EpiBf16 ep{(bf16*)t.act[1], net.b[1], 1, rows, 1 << 30, 0, N};
      TC_TRY((gemm<64, 2, false, false>(A, Bw, ep, rows, Kl, 1, 1, Kl, any, st)));
    } else if (l == 2) {
      const EpiBf16 ep{(bf16*)t.act[2], net.b[2], 1, rows, 1 << 30, 0, N};
      TC_TRY((gemm<128, 3, false, false>(A, Bw, ep, rows, Kl, 1, 1, Kl, any, st)));
    } else {  // the last convolution writes the dense layer's feature rows ((y, x, c) order, pitch 8200)
      const EpiBf16 ep{(bf16*)t.feat, net.b[3], 1, rows, 64, kFeatPitch, N};
      TC_TRY((gemm<128, 4, false, false>(A, Bw, ep, rows, Kl, 1, 1, Kl, any, st)));
    }
  }
  k_feat_tail<<<(B * (kFeatPitch - kFeat) + 255) / 256, 256, 0, st>>>((bf16*)t.feat, cs, B);
  note_launches(1);
  // dense layer: K = 8200 split 16 ways into FP32 partials, then summed with bias and ReLU
  const int Z = 16, kc = chunk_of(kFeatPitch, Z);
  const EpiF32 ep{t.part, (long long)B * kHid, B, kHid};
  TC_TRY((gemm<128, 4, false, false>(PlainK{(const bf16*)t.feat, kFeatPitch, B}, PlainK{(const bf16*)t.w1b, kFeatPitch, kHid},
                                  ep, B, kFeatPitch, 1, Z, kc, any, st)));
  k_sum_z<<<(unsigned)(((long long)B * kHid + 31) / 32), 256, 0, st>>>(t.part, Z, (long long)B * kHid, net.b1, kHid, h);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t cnn_tc_backward(int B, const CnnTc& t, const float* dh, const CnnGrad& g, cudaStream_t st) {
  const void* any = t.wb[1];
  (void)dh;  // its BF16 copy t.dhb, written with it, is what the GEMMs read
  const cudaError_t ez = cudaMemsetAsync(t.tickets, 0, kColTickets * sizeof(unsigned), st);
  if (ez != cudaSuccess) return ez;
  // dense layer: dW1[n][f] = sum_b dh[b][n] feat[b][f] (rows f, both operands MN-major)
  TC_TRY((gemm<128, 3, true, true>(PlainMN{(const bf16*)t.feat, kFeatPitch, kFeatPitch}, PlainMN{(const bf16*)t.dhb, kHid, kHid},
                                EpiF32T{g.w1, 0, kFeat + 2, kFeat + 2}, kFeatPitch, B, 1, 1, B, any, st)));
  // ... and dfeat[b][f] = sum_n dh[b][n] W1[n][f] (rows b, B MN-major) -> dY of the last convolution
  // (masked, BF16) and its per-channel column sums
  const int nmt = (B + kBM - 1) / kBM;
  TC_TRY((gemm<128, 2, false, true>(PlainK{(const bf16*)t.dhb, kHid, B}, PlainMN{(const bf16*)t.w1b, kFeatPitch, kFeat},
                                    EpiDfeat{(bf16*)t.dy3, (const bf16*)t.feat, t.colpart, B}, B, kHid, kFeat / 128, 1,
                                    kHid, any, st)));
  TC_TRY(colreduce(t.colpart, (kFeat / 128) * nmt, 128, 128, g.b[3], t.part, t.tickets, st));
  // convolutions 3, 2, 1: weight gradient (split over pixels), then the data gradient of the layer below
  const bf16* dyl = (const bf16*)t.dy3;
  for (int l = 3; l >= 1; --l) {
    const int H = kEdge[l], lwo = l == 1 ? 5 : (l == 2 ? 4 : 3), lc = l == 1 ? 5 : (l == 2 ? 6 : 7);
    const int ln = l == 1 ? 6 : 7;  // log2 N_l
    const int rows = B * kEdge[l + 1] * kEdge[l + 1], N = kCh[l + 1], Kl = 9 * kCh[l], C = kCh[l];
    const ConvGeomB geo{(const bf16*)t.act[l - 1], H, lwo, lc, rows, Kl};
    const int tiles = (Kl + kBM - 1) / kBM;
    const int Z = dw_splits(tiles, rows, t.part_floats, (long long)N * Kl);
    const int kc = chunk_of(rows, Z);
    const EpiF32T epw{t.part, (long long)N * Kl, Kl, Kl};
    if (N == 64)
      TC_TRY((gemm<64, 3, true, true>(ConvMN{geo}, PlainMN{dyl, N, N}, epw, Kl, rows, 1, Z, kc, any, st)));
    else
      TC_TRY((gemm<128, 4, true, true>(ConvMN{geo}, PlainMN{dyl, N, N}, epw, Kl, rows, 1, Z, kc, any, st)));
    k_sum_z<<<(unsigned)(((long long)N * Kl + 31) / 32), 256, 0, st>>>(t.part, Z, (long long)N * Kl, nullptr, 1, g.w[l]);
    note_launches(1);
    // data gradient, four parity classes in one launch; output dY of conv l - 1 and its bias partials
    bf16* dyo = (bf16*)(l == 2 ? t.dy[1] : t.dy[0]);
    const ParityK A{dyl, lwo, ln, rows};
    const ClassWt Bw{(const bf16*)t.wt[l], ln, C};
    if (C == 128)
      TC_TRY((gemm<128, 3, false, false>(A, Bw, EpiDx<128>{dyo, (const bf16*)t.act[l - 1], t.colpart, lwo, H, rows}, rows,
                                      9 * N, 1, 4, 1 << 30, any, st)));
    else if (C == 64)
      TC_TRY((gemm<64, 2, false, false>(A, Bw, EpiDx<64>{dyo, (const bf16*)t.act[l - 1], t.colpart, lwo, H, rows}, rows,
                                     9 * N, 1, 4, 1 << 30, any, st)));
    else
      TC_TRY((gemm<32, 2, false, false>(A, Bw, EpiDx<32>{dyo, (const bf16*)t.act[l - 1], t.colpart, lwo, H, rows}, rows,
                                     9 * N, 1, 4, 1 << 30, any, st)));
    TC_TRY(colreduce(t.colpart, 4 * ((rows + kBM - 1) / kBM), C, C, g.b[l - 1], t.part, t.tickets, st));
    dyl = dyo;
  }
  // the first convolution's weight gradient on the SIMT pipes
  const int G = kConv0Ctas;
  k_conv0_dw<<<G, 256, 0, st>>>(dyl, (const bf16*)t.imgb, B * 4096, t.colpart);
  note_launches(1);
  TC_TRY(colreduce(t.colpart, G, 288, 288, g.w[0], t.part, t.tickets, st));
  return cudaGetLastError();
}

}  // namespace digs
