// Weight-predictor CNN: a downsampled projection (128 x 128) and its gantry angle -> the projection's R
// low-rank temporal weights, used as the warm start of the per-projection weights of a reconstruction.
// (Not part of the paper; it learns the inverse of the forward model from pairs the forward model
// renders.)
//
// Network: four 3 x 3 convolutions of stride 2 and padding 1 (1 -> 32 -> 64 -> 128 -> 128 channels,
// 128^2 -> 64^2 -> 32^2 -> 16^2 -> 8^2), each followed by ReLU; the 8 x 8 x 128 features and
// (cos theta, sin theta) feed a 128-unit ReLU layer and a linear layer to R outputs.  Activations are
// NHWC; a convolution is im2col (rows = output pixels, columns = (ky, kx, c)) times the transposed
// weight matrix W[Co][ky][kx][Ci], so every layer, forward and backward, is one of three GEMM forms:
//   forward      Y[M][N]  = X[M][K] W[N][K]^T      (+ bias, ReLU)
//   data grad    dX[M][K] = dY[M][N] W[N][K]
//   weight grad  dW[N][K] = dY[M][N]^T X[M][K]     (split over M, partials summed in a fixed order)
// The forward and backward run either in FP32 on the SIMT pipes or, with DIGS_CNN_TENSOR_CORES, with the
// large GEMMs (the convolutions and the 8194-wide layer) on the tensor cores: BF16 operands rounded from
// the FP32 activations, gradients and weights, FP32 accumulation; the R-wide output layer stays FP32.
// Inference reads BF16 weights and activations and runs its large GEMMs on the tensor cores.
#include <cuda_bf16.h>

#include <algorithm>

#include "digs_internal.h"

namespace digs {

namespace {

constexpr int kConvs = 4;
constexpr int kCh[kConvs + 1] = {1, 32, 64, 128, 128};
constexpr int kEdge[kConvs + 1] = {128, 64, 32, 16, 8};
constexpr int kFeat = 8 * 8 * 128;
constexpr int kFeatIn = kFeat + 2;
constexpr int kHid = 128;
constexpr int kMaxBatch = 1024;

struct ParamOffsets {
  size_t w[kConvs], b[kConvs], w1, b1, w2, b2, total;
};

ParamOffsets param_offsets(int R) {
  ParamOffsets o;
  size_t off = 0;
  for (int l = 0; l < kConvs; ++l) {
    o.w[l] = off;
    off += (size_t)kCh[l + 1] * 9 * kCh[l];
    o.b[l] = off;
    off += kCh[l + 1];
  }
  o.w1 = off;
  off += (size_t)kHid * kFeatIn;
  o.b1 = off;
  off += kHid;
  o.w2 = off;
  off += (size_t)R * kHid;
  o.b2 = off;
  off += R;
  o.total = off;
  return o;
}

size_t rows(int l, int B) { return (size_t)B * kEdge[l + 1] * kEdge[l + 1]; }  // output pixels of conv l
size_t kdim(int l) { return (size_t)9 * kCh[l]; }

// Workspace of one batch: activations for the backward, gradients, split-K partials, BF16 copies.
struct CnnWs {
  float *col[kConvs], *act[kConvs], *feat, *h, *out, *dout, *dh, *dfeat, *dact0, *dact1, *dcol, *part, *loss;
  CnnTc tc;  // the tensor-core path's BF16 activations, gradients and weight copies (cnn_tc.cu)
  size_t bytes;
};

constexpr int kSplits = 32;

// Floats of the split-K partial buffer: 32 splits of the largest dW (128 x 1152) or 16 splits of the
// B x 128 hidden layer, whichever is more.
long long part_floats(int B) {
  return std::max<long long>((long long)kSplits * 128 * 1152, 16LL * B * 128);
}

CnnWs cnn_layout(void* base, int B, int R) {
  CnnWs w;
  size_t off = 0;
  char* p = (char*)base;
  auto take = [&](size_t bytes) -> char* {
    char* q = p ? p + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return q;
  };
  size_t max_act = 0, max_col = 0;
  for (int l = 0; l < kConvs; ++l) {
    w.col[l] = (float*)take(rows(l, B) * kdim(l) * 4);
    w.act[l] = (float*)take(rows(l, B) * kCh[l + 1] * 4);
    max_act = std::max(max_act, rows(l, B) * kCh[l + 1]);
    max_col = std::max(max_col, rows(l, B) * kdim(l));
  }
  max_act = std::max(max_act, (size_t)B * kFeatIn);
  w.feat = (float*)take((size_t)B * kFeatIn * 4);
  w.h = (float*)take((size_t)B * kHid * 4);
  w.out = (float*)take((size_t)B * R * 4 + 4);
  w.dout = (float*)take((size_t)B * R * 4 + 4);
  w.dh = (float*)take((size_t)B * kHid * 4);
  w.dfeat = (float*)take((size_t)B * kFeatIn * 4);
  w.dact0 = (float*)take(max_act * 4);
  w.dact1 = (float*)take(max_act * 4);
  w.dcol = (float*)take(max_col * 4);
  w.part = (float*)take((size_t)part_floats(B) * 4);  // split-K and bias partials
  w.loss = (float*)take(256);
  off += cnn_tc_layout(p ? p + off : nullptr, B, &w.tc);
  w.bytes = off;
  return w;
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// C(m, n) = sum_k A(m, k) B(k, n) over this block's k-range; A(m, k) = AT ? A[k lda + m] : A[m lda + k],
// B(k, n) = BT ? B[n ldb + k] : B[k ldb + n].  64 x 64 tile per 256 threads (4 x 4 per thread), 16-deep
// k slices in shared memory.  gridDim.z > 1: block z sums k in [z kchunk, (z + 1) kchunk) and writes its
// partial to C + z * zstride (summed later); else the epilogue adds bias[n] and applies ReLU if asked.
template <bool AT, bool BT, typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const TA* __restrict__ A, int lda,
                                              const TB* __restrict__ B, int ldb, TC* __restrict__ C, int ldc,
                                              int kchunk, long long zstride, const float* __restrict__ bias,
                                              int relu) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int t = threadIdx.x + 256 * e;  // 1024 elements of each 64 x 16 slice
      int mm, kk;
      if (AT) { kk = t >> 6; mm = t & 63; } else { mm = t >> 4; kk = t & 15; }
      const int m = m0 + mm, k = k0 + kk;
      float a = 0.f;
      if (m < M && k < ke) a = to_f(AT ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]);
      As[kk][mm] = a;
      int nn, kk2;
      if (BT) { nn = t >> 4; kk2 = t & 15; } else { kk2 = t >> 6; nn = t & 63; }
      const int n = n0 + nn, k2 = k0 + kk2;
      float bv = 0.f;
      if (n < N && k2 < ke) bv = to_f(BT ? B[(size_t)n * ldb + k2] : B[(size_t)k2 * ldb + n]);
      Bs[kk2][nn] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  TC* Cz = C + (size_t)blockIdx.z * zstride;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (gridDim.z == 1) {
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
      }
      Cz[(size_t)m * ldc + n] = from_f<TC>(v);
    }
  }
}

template <bool AT, bool BT, typename TA, typename TB, typename TC>
cudaError_t gemm(int M, int N, int K, const TA* A, int lda, const TB* B, int ldb, TC* C, int ldc, const float* bias,
                 bool relu, cudaStream_t st, int splits = 1, long long zstride = 0) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
  k_gemm<AT, BT, TA, TB, TC><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, kchunk, zstride, bias,
                                                   relu ? 1 : 0);
  note_launches(1);
  return cudaGetLastError();
}

// The R-wide output layer, FP32: out[b][r] = b2[r] + sum_n h[b][n] W2[r][n], one warp per batch entry.
__global__ void __launch_bounds__(256) k_fc2_fwd(const float* __restrict__ h, const float* __restrict__ w2,
                                                 const float* __restrict__ b2, int B, int R, float* __restrict__ out) {
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= B) return;  // whole warps
  float x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = h[(size_t)b * kHid + lane + 32 * q];
  for (int r = 0; r < R; ++r) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) s = fmaf(x[q], w2[r * kHid + lane + 32 * q], s);
    s = warp_sum(s);
    if (lane == 0) out[(size_t)b * R + r] = s + b2[r];
  }
}

// Its parameter gradient, per block of batch entries (blockIdx.x selects entries b = blockIdx.x,
// blockIdx.x + gridDim.x, ...): part[block][r kHid + n] = sum_b dout[b][r] h[b][n] (threads n < kHid) and
// part[block][R kHid + r] = sum_b dout[b][r] (threads kHid + r); the blocks are added in order after.
__global__ void __launch_bounds__(kHid + 32) k_fc2_wgrad(const float* __restrict__ dout, const float* __restrict__ h,
                                                         int B, int R, float* __restrict__ part) {
  const int n = threadIdx.x;
  float acc[DIGS_MAX_R] = {0.f, 0.f, 0.f, 0.f};
  if (n < kHid) {
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
      const float x = h[(size_t)b * kHid + n];
#pragma unroll
      for (int r = 0; r < DIGS_MAX_R; ++r)
        if (r < R) acc[r] = fmaf(dout[(size_t)b * R + r], x, acc[r]);
    }
    for (int r = 0; r < R; ++r) part[(size_t)blockIdx.x * (R * kHid + R) + r * kHid + n] = acc[r];
  } else if (n - kHid < R) {
    const int r = n - kHid;
    float t = 0.f;
    for (int b = blockIdx.x; b < B; b += gridDim.x) t += dout[(size_t)b * R + r];
    part[(size_t)blockIdx.x * (R * kHid + R) + R * kHid + r] = t;
  }
}

// dh[b][n] = [h[b][n] > 0] sum_r dout[b][r] W2[r][n]: the gradient of the dense layer's pre-activation.
// dh = dL/d(dense pre-activation), masked by the dense layer's ReLU; with dhb, also its BF16 copy (the
// tensor-core backward's operand).
__global__ void k_fc2_dh(const float* __restrict__ dout, const float* __restrict__ w2, const float* __restrict__ h,
                         int B, int R, float* __restrict__ dh, uint16_t* __restrict__ dhb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * kHid) return;
  const int b = i / kHid, n = i - b * kHid;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s = fmaf(dout[(size_t)b * R + r], w2[r * kHid + n], s);
  const float v = h[i] > 0.f ? s : 0.f;
  dh[i] = v;
  if (dhb) dhb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// out[i] (+)= sum_z part[z][i], z in a fixed order.
__global__ void k_sum_splits(const float* __restrict__ part, int splits, long long n, float* __restrict__ out,
                             int accumulate) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = accumulate ? out[i] : 0.f;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * n + i];
  out[i] = s;
}

// db[n] = sum_m dY[m][n]: each block sums 32 columns over a slice of rows (lane = column), then the
// slices are summed in order.
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ dY, int M, int N, int rows_per,
                                                float* __restrict__ part) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + lane;
  const int m0 = blockIdx.y * rows_per, m1 = min(M, m0 + rows_per);
  float s = 0.f;
  if (n < N)
    for (int m = m0 + warp; m < m1; m += 8) s += dY[(size_t)m * N + n];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && n < N) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    part[(size_t)blockIdx.y * N + n] = t;
  }
}

cudaError_t colsum(const float* dY, int M, int N, float* part, float* db, cudaStream_t st) {
  // about 4096 rows per slice (at least kSplits slices), so that tall thin dY fill the GPU
  const int splits = std::max(kSplits, std::min((M + 4095) / 4096, 1024));
  const int rows_per = (M + splits - 1) / splits;
  dim3 grid((N + 31) / 32, splits);
  k_colsum<<<grid, 256, 0, st>>>(dY, M, N, rows_per, part);
  k_sum_splits<<<(N + 255) / 256, 256, 0, st>>>(part, splits, N, db, 0);
  note_launches(2);
  return cudaGetLastError();
}

// col[(b Ho + y) Wo + x][(ky 3 + kx) C + c] = in[b][2y + ky - 1][2x + kx - 1][c] (0 outside), NHWC.
template <typename TI, typename TO>
__global__ void k_im2col(const TI* __restrict__ in, int B, int H, int W, int C, TO* __restrict__ col) {
  const int Ho = H / 2, Wo = W / 2, K = 9 * C;
  const long long total = (long long)B * Ho * Wo * K;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % K);
    const long long r = i / K;
    const int x = (int)(r % Wo), y = (int)((r / Wo) % Ho), b = (int)(r / ((long long)Wo * Ho));
    const int c = k % C, tap = k / C, ky = tap / 3, kx = tap % 3;
    const int iy = 2 * y + ky - 1, ix = 2 * x + kx - 1;
    float v = 0.f;
    if (iy >= 0 && iy < H && ix >= 0 && ix < W) v = to_f(in[(((size_t)b * H + iy) * W + ix) * C + c]);
    col[i] = from_f<TO>(v);
  }
}

// din[b][iy][ix][c] = sum over the taps that read it of dcol[(b Ho + y) Wo + x][(ky 3 + kx) C + c].
__global__ void k_col2im(const float* __restrict__ dcol, int B, int H, int W, int C, float* __restrict__ din) {
  const int Ho = H / 2, Wo = W / 2, K = 9 * C;
  const long long total = (long long)B * H * W * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long r = i / C;
    const int ix = (int)(r % W), iy = (int)((r / W) % H), b = (int)(r / ((long long)W * H));
    float s = 0.f;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int ty = iy + 1 - ky;
      if (ty < 0 || (ty & 1) || (ty >> 1) >= Ho) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int tx = ix + 1 - kx;
        if (tx < 0 || (tx & 1) || (tx >> 1) >= Wo) continue;
        s += dcol[(((size_t)b * Ho + (ty >> 1)) * Wo + (tx >> 1)) * K + (ky * 3 + kx) * C + c];
      }
    }
    din[i] = s;
  }
}

unsigned grid_for(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32); }

// feat[b] = (act3[b] (8192 values), cos theta_b, sin theta_b)
template <typename TI, typename TO>
__global__ void k_features(const TI* __restrict__ act3, const float* __restrict__ cs, int B, TO* __restrict__ feat) {
  const long long total = (long long)B * kFeatIn;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / kFeatIn), j = (int)(i % kFeatIn);
    const float v = j < kFeat ? to_f(act3[(size_t)b * kFeat + j]) : cs[2 * b + (j - kFeat)];
    feat[i] = from_f<TO>(v);
  }
}

// dact3[b][j] = dfeat[b][j] for the image features (the angle inputs get no gradient).
__global__ void k_feat_grad(const float* __restrict__ dfeat, int B, float* __restrict__ dact3) {
  const long long total = (long long)B * kFeat;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    dact3[i] = dfeat[(i / kFeat) * kFeatIn + i % kFeat];
}

// dY *= [Y > 0] (ReLU backward; Y is the post-activation value).
__global__ void k_relu_bwd(const float* __restrict__ Y, long long n, float* __restrict__ dY) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(Y[i] > 0.f)) dY[i] = 0.f;
}

// loss = mean (out - target)^2 over B x R; dout = 2 (out - target) / (B R).  One block.
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ out, const float* __restrict__ target, int n,
                                             float* __restrict__ dout, float* __restrict__ loss) {
  __shared__ float red[8];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float r = out[i] - target[i];
    dout[i] = 2.f * r / (float)n;
    s = fmaf(r, r, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k];
    *loss = t / (float)n;
  }
}

// The network input [B][128][128] of a projection stack [B][nv][nu], times `scale`: the 2 x 2 means of
// 256 x 256 projections, or 128 x 128 projections as they are.
__global__ void k_downsample(const float* __restrict__ proj, int B, int nu, int nv, float scale,
                             float* __restrict__ img) {
  const int f = nu / 128;  // 2: 2 x 2 means of a 256 x 256 projection; 1: a 128 x 128 one, scaled
  const long long total = (long long)B * 128 * 128;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % 128), y = (int)((i / 128) % 128), b = (int)(i / (128LL * 128));
    const float* p = proj + ((size_t)b * nv + f * y) * nu + f * x;
    img[i] = f == 2 ? 0.25f * scale * (p[0] + p[1] + p[nu] + p[nu + 1]) : scale * p[0];
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// He-normal weights (std sqrt(2 / fan_in)) from a counter-based generator (splitmix64 of seed and index,
// Box-Muller), zero biases.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_init(float* __restrict__ p, long long n, unsigned long long seed, float std_dev, int is_bias) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (is_bias) { p[i] = 0.f; continue; }
    const unsigned long long r = splitmix64(seed ^ splitmix64((unsigned long long)i));
    const float u1 = ((float)(r >> 40) + 1.f) * (1.f / 16777217.f);          // (0, 1]
    const float u2 = (float)((r >> 16) & 0xFFFFFFull) * (1.f / 16777216.f);  // [0, 1)
    p[i] = std_dev * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
  }
}

template <typename T>
struct NetPtrs {  // one precision's view of the parameters
  const T *w[kConvs], *w1, *w2;
  const float *b[kConvs], *b1, *b2;
};

template <typename T>
NetPtrs<T> net_ptrs(const T* wp, const float* bp, const ParamOffsets& o) {
  NetPtrs<T> n;
  for (int l = 0; l < kConvs; ++l) {
    n.w[l] = wp + o.w[l];
    n.b[l] = bp + o.b[l];
  }
  n.w1 = wp + o.w1;
  n.b1 = bp + o.b1;
  n.w2 = wp + o.w2;
  n.b2 = bp + o.b2;
  return n;
}

#define CNN_TRY(...)                         \
  do {                                       \
    cudaError_t e__ = (__VA_ARGS__);         \
    if (e__ != cudaSuccess) return e__;      \
  } while (0)

CnnNet cnn_net(const NetPtrs<float>& N) {
  CnnNet n;
  for (int l = 0; l < kConvs; ++l) {
    n.w[l] = N.w[l];
    n.b[l] = N.b[l];
  }
  n.w1 = N.w1;
  n.b1 = N.b1;
  return n;
}

// Forward keeping every activation in the workspace for the backward.  tc: the tensor-core path of
// cnn_tc.cu up to the dense layer's output (BF16 activations), else FP32 SIMT GEMMs over im2col
// matrices; the R-wide output layer is FP32 either way.
cudaError_t forward_f32(const NetPtrs<float>& N, int R, const float* img, const float* cs, int B, const CnnWs& w,
                        bool tc, cudaStream_t st) {
  if (tc) {
    CNN_TRY(cnn_tc_forward(cnn_net(N), img, cs, B, w.tc, w.h, st));
  } else {
    const float* in = img;
    for (int l = 0; l < kConvs; ++l) {
      const int H = kEdge[l], C = kCh[l];
      const long long ncol = (long long)rows(l, B) * kdim(l);
      k_im2col<float, float><<<grid_for(ncol), 256, 0, st>>>(in, B, H, H, C, w.col[l]);
      note_launches(1);
      CNN_TRY(gemm<false, true>((int)rows(l, B), kCh[l + 1], (int)kdim(l), w.col[l], (int)kdim(l), N.w[l],
                                (int)kdim(l), w.act[l], kCh[l + 1], N.b[l], true, st));
      in = w.act[l];
    }
    k_features<float, float><<<grid_for((long long)B * kFeatIn), 256, 0, st>>>(w.act[kConvs - 1], cs, B, w.feat);
    note_launches(1);
    CNN_TRY(gemm<false, true>(B, kHid, kFeatIn, w.feat, kFeatIn, N.w1, kFeatIn, w.h, kHid, N.b1, true, st));
  }
  k_fc2_fwd<<<(B + 7) / 8, 256, 0, st>>>(w.h, N.w2, N.b2, B, R, w.out);
  note_launches(1);
  return cudaGetLastError();
}

// Backward of forward_f32 for dL/dout in w.dout; writes every parameter gradient to grad (layout as params).
cudaError_t backward_f32(const NetPtrs<float>& N, const ParamOffsets& o, int R, int B, const CnnWs& w, float* grad,
                         bool tc, cudaStream_t st) {
  // output layer
  constexpr int kFc2Blocks = 16;
  k_fc2_wgrad<<<kFc2Blocks, kHid + 32, 0, st>>>(w.dout, w.h, B, R, w.part);
  k_sum_splits<<<(R * kHid + R + 255) / 256, 256, 0, st>>>(w.part, kFc2Blocks, R * kHid + R, grad + o.w2, 0);
  k_fc2_dh<<<(B * kHid + 255) / 256, 256, 0, st>>>(w.dout, N.w2, w.h, B, R, w.dh, tc ? w.tc.dhb : nullptr);
  note_launches(3);
  CNN_TRY(colsum(w.dh, B, kHid, w.part, grad + o.b1, st));
  if (tc) {
    CnnGrad g;
    for (int l = 0; l < kConvs; ++l) {
      g.w[l] = grad + o.w[l];
      g.b[l] = grad + o.b[l];
    }
    g.w1 = grad + o.w1;
    return cnn_tc_backward(B, w.tc, w.dh, g, st);
  }
  // hidden layer
  CNN_TRY(gemm<true, false>(kHid, kFeatIn, B, w.dh, kHid, w.feat, kFeatIn, grad + o.w1, kFeatIn, nullptr, false, st));
  CNN_TRY(gemm<false, false>(B, kFeatIn, kHid, w.dh, kHid, N.w1, kFeatIn, w.dfeat, kFeatIn, nullptr, false, st));
  k_feat_grad<<<grid_for((long long)B * kFeat), 256, 0, st>>>(w.dfeat, B, w.dact0);
  note_launches(1);
  // convolutions, last to first; dact0 holds dL/d(output of conv l)
  float* dY = w.dact0;
  float* dX = w.dact1;
  for (int l = kConvs - 1; l >= 0; --l) {
    const int M = (int)rows(l, B), Nn = kCh[l + 1], K = (int)kdim(l);
    k_relu_bwd<<<grid_for((long long)M * Nn), 256, 0, st>>>(w.act[l], (long long)M * Nn, dY);
    note_launches(1);
    const long long ndw = (long long)Nn * K;
    const int splits = kSplits;  // split the B x H x W rows: dW is at most 128 x 1152
    CNN_TRY(gemm<true, false>(Nn, K, M, dY, Nn, w.col[l], K, w.part, K, nullptr, false, st, splits, ndw));
    k_sum_splits<<<(unsigned)((ndw + 255) / 256), 256, 0, st>>>(w.part, splits, ndw, grad + o.w[l], 0);
    note_launches(1);
    CNN_TRY(colsum(dY, M, Nn, w.part, grad + o.b[l], st));
    if (l > 0) {
      CNN_TRY(gemm<false, false>(M, K, Nn, dY, Nn, N.w[l], K, w.dcol, K, nullptr, false, st));
      const int H = kEdge[l], C = kCh[l];
      k_col2im<<<grid_for((long long)B * H * H * C), 256, 0, st>>>(w.dcol, B, H, H, C, dX);
      note_launches(1);
      float* t = dY;
      dY = dX;
      dX = t;
    }
  }
  return cudaGetLastError();
}

bool args_ok(int R, int B) { return R >= 1 && R <= DIGS_MAX_R && B >= 1 && B <= kMaxBatch; }

}  // namespace
}  // namespace digs

using namespace digs;

extern "C" {

size_t digs_cnn_params(int R) { return (R >= 1 && R <= DIGS_MAX_R) ? param_offsets(R).total : 0; }

size_t digs_cnn_workspace_size(int B, int R) { return args_ok(R, B) ? cnn_layout(nullptr, B, R).bytes : 0; }

digs_status digs_cnn_init(float* params, int R, unsigned long long seed, void* stream) {
  if (!params || R < 1 || R > DIGS_MAX_R) return DIGS_ERR_ARG;
  const ParamOffsets o = param_offsets(R);
  cudaStream_t st = (cudaStream_t)stream;
  auto init = [&](size_t off, long long n, int fan_in, int is_bias) {
    k_init<<<grid_for(n), 256, 0, st>>>(params + off, n, seed + off, sqrtf(2.f / (float)fan_in), is_bias);
    note_launches(1);
  };
  for (int l = 0; l < kConvs; ++l) {
    init(o.w[l], (long long)kCh[l + 1] * kdim(l), (int)kdim(l), 0);
    init(o.b[l], kCh[l + 1], 1, 1);
  }
  init(o.w1, (long long)kHid * kFeatIn, kFeatIn, 0);
  init(o.b1, kHid, 1, 1);
  init(o.w2, (long long)R * kHid, kHid, 0);
  init(o.b2, R, 1, 1);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

digs_status digs_cnn_prepare_input(const float* proj, int B, int nu, int nv, float scale, float* img, void* stream) {
  if (!proj || !img || B < 1 || nu != nv || (nu != 256 && nu != 128)) return DIGS_ERR_ARG;
  k_downsample<<<grid_for((long long)B * 128 * 128), 256, 0, (cudaStream_t)stream>>>(proj, B, nu, nv, scale, img);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

digs_status digs_cnn_forward(const float* params, int R, const float* img, const float* cs, int B, float* w_out,
                             int flags, void* ws, size_t ws_bytes, void* stream) {
  if (!params || !img || !cs || !w_out || !ws || !args_ok(R, B)) return DIGS_ERR_ARG;
  const CnnWs w = cnn_layout(ws, B, R);
  if (w.bytes > ws_bytes) return DIGS_ERR_ARG;
  const ParamOffsets o = param_offsets(R);
  cudaStream_t st = (cudaStream_t)stream;
  const bool tc = (flags & DIGS_CNN_TENSOR_CORES) != 0;
  if (forward_f32(net_ptrs<float>(params, params, o), R, img, cs, B, w, tc, st) != cudaSuccess) return DIGS_ERR_CUDA;
  if (cudaMemcpyAsync(w_out, w.out, (size_t)B * R * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return DIGS_ERR_CUDA;
  return DIGS_OK;
}

digs_status digs_cnn_backward(const float* params, int R, int B, const float* grad_w, float* grad_params, int flags,
                              void* ws, size_t ws_bytes, void* stream) {
  if (!params || !grad_w || !grad_params || !ws || !args_ok(R, B)) return DIGS_ERR_ARG;
  const CnnWs w = cnn_layout(ws, B, R);
  if (w.bytes > ws_bytes) return DIGS_ERR_ARG;
  const ParamOffsets o = param_offsets(R);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(w.dout, grad_w, (size_t)B * R * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return DIGS_ERR_CUDA;
  const bool tc = (flags & DIGS_CNN_TENSOR_CORES) != 0;
  if (backward_f32(net_ptrs<float>(params, params, o), o, R, B, w, grad_params, tc, st) != cudaSuccess)
    return DIGS_ERR_CUDA;
  return DIGS_OK;
}

digs_status digs_cnn_train_step(float* params, float* m, float* v, float* grad, int step, float lr, int R,
                                const float* img, const float* cs, const float* target, int B, float* loss_out,
                                int flags, void* ws, size_t ws_bytes, void* stream) {
  if (!params || !m || !v || !grad || !img || !cs || !target || !loss_out || !ws || step < 1 || !args_ok(R, B))
    return DIGS_ERR_ARG;
  const CnnWs w = cnn_layout(ws, B, R);
  if (w.bytes > ws_bytes) return DIGS_ERR_ARG;
  const ParamOffsets o = param_offsets(R);
  cudaStream_t st = (cudaStream_t)stream;
  const NetPtrs<float> N = net_ptrs<float>(params, params, o);
  const bool tc = (flags & DIGS_CNN_TENSOR_CORES) != 0;
  if (forward_f32(N, R, img, cs, B, w, tc, st) != cudaSuccess) return DIGS_ERR_CUDA;
  k_mse<<<1, 256, 0, st>>>(w.out, target, B * R, w.dout, loss_out);
  note_launches(1);
  if (backward_f32(N, o, R, B, w, grad, tc, st) != cudaSuccess) return DIGS_ERR_CUDA;
  AdamGroup g{params, grad, m, v, (long long)o.total, 0, 0, lr, lr};
  if (launch_adam(&g, 1, 0.9f, 0.999f, 1e-8f, step, nullptr, 0, st) != cudaSuccess) return DIGS_ERR_CUDA;
  return DIGS_OK;
}

digs_status digs_cnn_infer_bf16(const float* params, int R, const float* img, const float* cs, int B, float* w_out,
                                void* ws, size_t ws_bytes, void* stream) {
  if (!params || !img || !cs || !w_out || !ws || !args_ok(R, B)) return DIGS_ERR_ARG;
  const CnnWs w = cnn_layout(ws, B, R);
  if (w.bytes > ws_bytes) return DIGS_ERR_ARG;
  const ParamOffsets o = param_offsets(R);
  cudaStream_t st = (cudaStream_t)stream;
  const NetPtrs<float> N = net_ptrs<float>(params, params, o);
  if (cnn_tc_forward(cnn_net(N), img, cs, B, w.tc, w.h, st) != cudaSuccess) return DIGS_ERR_CUDA;
  k_fc2_fwd<<<(B + 7) / 8, 256, 0, st>>>(w.h, N.w2, N.b2, B, R, w_out);
  note_launches(1);
  if (cudaGetLastError() != cudaSuccess) return DIGS_ERR_CUDA;
  return DIGS_OK;
}

}  // extern "C"
