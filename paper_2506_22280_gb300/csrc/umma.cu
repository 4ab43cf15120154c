// Dense GEMM on the fifth-generation tensor cores (tcgen05, sm_103a): C = op(A) op(B) with BF16 operands
// and FP32 accumulation in tensor memory, behind digs_gemm_bf16 (FP32 operands rounded while staged).
// The CNN's own layers run on the kernels of cnn_tc.cu, which read BF16 activations in place.
//
// C(m, n) = sum_k A(m, k) B(k, n); A(m, k) = AT ? A[k lda + m] : A[m lda + k] and
// B(k, n) = BT ? B[n ldb + k] : B[k ldb + n], FP32 in global memory.  One CTA of 128 threads per
// 128 x 64 tile of C:
//   * all four warps stage 64-deep K slices of A (128 x 64) and B (64 x 64) into shared memory,
//     rounding to BF16 (round to nearest even) and writing the K-major, non-swizzled layout the tensor
//     core reads: 8-row x 16-byte core matrices, core matrix (row group g, k chunk kc) at
//     (8 g + kc) 128 bytes, so that 8-row groups lie 1024 bytes apart and K chunks 128 bytes apart;
//   * one thread issues four 128 x 64 x 16 tcgen05.mma per slice into a 128-lane x 64-column FP32
//     accumulator in tensor memory and commits them to the slice's mbarrier; the slice buffers are
//     double-buffered, so staging slice k + 1 overlaps the MMAs of slice k;
//   * each warp reads its 32 accumulator lanes (rows) back with tcgen05.ld, adds the bias and applies
//     ReLU when asked, and puts them in shared memory, from where whole rows go out with 16-byte stores.
// gridDim.z > 1 splits K: block z sums k in [z kchunk, (z + 1) kchunk) into C + z zstride (no bias).
// Every mbarrier wait is bounded; a wait of the K loop that gives up sets *status to 1, and the block
// still waits for its own MMAs (with the default bound, whatever digs_set_wait_limit says), frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "digs_internal.h"
#include "tcgen05.cuh"

namespace digs {
namespace {

constexpr int kTcThreads = 128;
constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kStageA = kBM * kBK * 2;  // bytes of one A slice (16 KB)
constexpr int kStageB = kBN * kBK * 2;  // bytes of one B slice (8 KB)
constexpr int kTmemCols = 64;           // FP32 accumulator columns (= kBN)
constexpr size_t kTcSmem = 1024 + 2 * kStageA + 2 * kStageB + 64;  // 1 KB alignment slack, buffers, barriers
constexpr unsigned kWaitLimit = tc::kWaitLimit;

// Tests a K-loop mbarrier wait makes before it gives up (digs_set_wait_limit; read at launch).
unsigned g_loop_wait_limit = kWaitLimit;

using tc::fence_after;
using tc::fence_async_smem;
using tc::fence_before;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::smem_desc;
using tc::smem_u32;
using tc::tmem_ld16;

constexpr uint32_t kIdesc = tc::idesc_bf16(kBM, kBN, false, false);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  tc::mma_bf16(tmem_d, da, db, kIdesc, accumulate);
}

__device__ __forceinline__ float ld_f(const float* p) { return __ldg(p); }
__device__ __forceinline__ void st_c(float* p, float v) { *p = v; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void st_c4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// A whole 8-element chunk with 16-byte loads (vec: the operand's base and pitch allow them).
__device__ __forceinline__ uint4 load_vec8(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  return make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(b.x, b.y), pack_bf16(b.z, b.w));
}

// One 8-element K chunk of row `row` of an operand, K-range [k, k + 8) clipped to [.., kend), rows
// beyond `rows` zero; T (transposed) reads element (row, kk) at P[kk ld + row], else P[row ld + kk].
template <bool T, typename TP>
__device__ __forceinline__ uint4 load_chunk(const TP* __restrict__ P, int ld, int row, int rows, int k, int kend,
                                            bool vec) {
  if (!T && vec && row < rows && k + 8 <= kend) return load_vec8(P + (size_t)row * ld + k);
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int kk = k + e;
    x[e] = (row < rows && kk < kend) ? ld_f(T ? P + (size_t)kk * ld + row : P + (size_t)row * ld + kk) : 0.f;
  }
  return make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
}

// Stage the K slice [k0, k0 + 64) of the block's A rows and B columns.  Consecutive threads take
// consecutive K chunks when K is the contiguous global index, else consecutive rows.  Every chunk is
// loaded (and rounded) before any is stored, so that all of the thread's loads are in flight together.
template <bool AT, bool BT, typename TA, typename TB>
__device__ __forceinline__ void stage(const TA* __restrict__ A, int lda, const TB* __restrict__ B, int ldb, int M,
                                      int N, int m0, int n0, int k0, int kend, uint8_t* sA, uint8_t* sB, int vec) {
  constexpr int CA = (kBM * 8) / kTcThreads, CB = (kBN * 8) / kTcThreads;
  uint4 va[CA], vb[CB];
#pragma unroll
  for (int i = 0; i < CA; ++i) {
    const int c = threadIdx.x + i * kTcThreads;
    const int kc = AT ? c / kBM : c & 7, mm = AT ? c % kBM : c >> 3;
    va[i] = load_chunk<AT>(A, lda, m0 + mm, M, k0 + kc * 8, kend, (vec & 1) != 0);
  }
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const int c = threadIdx.x + i * kTcThreads;
    const int kc = BT ? c & 7 : c / kBN, nn = BT ? c >> 3 : c % kBN;
    vb[i] = load_chunk<!BT>(B, ldb, n0 + nn, N, k0 + kc * 8, kend, (vec & 2) != 0);
  }
#pragma unroll
  for (int i = 0; i < CA; ++i) {
    const int c = threadIdx.x + i * kTcThreads;
    const int kc = AT ? c / kBM : c & 7, mm = AT ? c % kBM : c >> 3;
    *reinterpret_cast<uint4*>(sA + ((mm >> 3) * 8 + kc) * 128 + (mm & 7) * 16) = va[i];
  }
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    const int c = threadIdx.x + i * kTcThreads;
    const int kc = BT ? c & 7 : c / kBN, nn = BT ? c >> 3 : c % kBN;
    *reinterpret_cast<uint4*>(sB + ((nn >> 3) * 8 + kc) * 128 + (nn & 7) * 16) = vb[i];
  }
}

template <bool AT, bool BT, typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(int M, int N, int K, const TA* __restrict__ A, int lda,
                                                        const TB* __restrict__ B, int ldb, TC* __restrict__ C,
                                                        int ldc, int kchunk, long long zstride,
                                                        const float* __restrict__ bias, int relu, int vec,
                                                        int* status, unsigned wait_limit) {
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = sm;
  uint8_t* sB = sm + 2 * kStageA;
  uint64_t* bar = (uint64_t*)(sB + 2 * kStageB);
  uint32_t* tslot = (uint32_t*)(bar + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int nk = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, kTmemCols);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  int ok = 1;
  int issued = 0;  // slices whose MMAs were committed
  for (int s = 0; s < nk; ++s) {
    const int buf = s & 1;
    if (s >= 2) ok = __syncthreads_and(ok && mbar_wait(bar + buf, (uint32_t)(((s >> 1) - 1) & 1), wait_limit));
    if (!ok) break;
    stage<AT, BT>(A, lda, B, ldb, M, N, m0, n0, kb + s * kBK, ke, sA + buf * kStageA, sB + buf * kStageB, vec);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      const uint32_t a0 = smem_u32(sA + buf * kStageA), b0 = smem_u32(sB + buf * kStageB);
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j) {
        // MMA j covers k chunks 2j and 2j + 1 (256 bytes in): K chunks 128 bytes apart, row groups 1024
        const uint64_t da = smem_desc(a0 + j * 256, 128, 1024);
        const uint64_t db = smem_desc(b0 + j * 256, 128, 1024);
        mma_bf16(tmem, da, db, (s > 0 || j > 0) ? 1u : 0u);
      }
      mma_commit(bar + buf);
    }
    issued = s + 1;
  }
  // the last commit tracks every MMA issued before it: always drained (default bound) before the tensor
  // memory is read or freed, and the outcome made block-uniform
  const bool drained = issued == 0 || mbar_wait(bar + ((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1), kWaitLimit);
  ok = __syncthreads_and(ok && drained);
  fence_after();
  // epilogue: accumulator lanes -> registers (+ bias, ReLU) -> the 128 x 64 tile in the (now idle)
  // staging buffers -> global rows, 4 consecutive columns per thread, 16 threads per row
  constexpr int TP = kBN + 4;  // tile row pitch in floats (16-byte aligned rows)
  float* tile = reinterpret_cast<float*>(sm);
  const int r = warp * 32 + lane;
#pragma unroll
  for (int c0 = 0; c0 < kBN; c0 += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n0 + c0 + j;
      float x = issued > 0 ? v[j] : 0.f;
      if (gridDim.z == 1 && n < N) {
        if (bias) x += bias[n];
        if (relu) x = fmaxf(x, 0.f);
      }
      v[j] = x;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(tile + r * TP + c0 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
  __syncthreads();
  TC* Cz = C + (size_t)blockIdx.z * zstride;
  const bool vec_c = (ldc % 4) == 0 && ((uintptr_t)Cz % (4 * sizeof(TC))) == 0;
  const int cq = (threadIdx.x & 15) * 4;
  if (ok) {
#pragma unroll 4
    for (int i = 0; i < kBM / 8; ++i) {
      const int rr = (threadIdx.x >> 4) + 8 * i, m = m0 + rr, n = n0 + cq;
      if (m >= M || n >= N) continue;
      const float4 x = *reinterpret_cast<const float4*>(tile + rr * TP + cq);
      TC* dst = Cz + (size_t)m * ldc + n;
      if (vec_c && n + 3 < N) {
        st_c4(dst, x);
      } else {
        st_c(dst, x.x);
        if (n + 1 < N) st_c(dst + 1, x.y);
        if (n + 2 < N) st_c(dst + 2, x.z);
        if (n + 3 < N) st_c(dst + 3, x.w);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  if (!ok && threadIdx.x == 0 && status) atomicExch(status, 1);
}

template <bool AT, bool BT, typename TA, typename TB, typename TC>
cudaError_t launch_tc(int M, int N, int K, const TA* A, int lda, const TB* B, int ldb, TC* C, int ldc,
                      const float* bias, bool relu, int splits, long long zstride, int* status, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<AT, BT, TA, TB, TC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (splits < 1) splits = 1;
  const int kchunk = ((K + splits - 1) / splits + kBK - 1) / kBK * kBK;
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splits);
  // 16-byte loads of whole K chunks where K is the contiguous index and base and pitch are aligned
  constexpr int per16a = 16 / (int)sizeof(TA), per16b = 16 / (int)sizeof(TB);
  const int vec = ((!AT && ((uintptr_t)A & 15) == 0 && lda % per16a == 0) ? 1 : 0) |
                  ((BT && ((uintptr_t)B & 15) == 0 && ldb % per16b == 0) ? 2 : 0);
  k_gemm_tc<AT, BT, TA, TB, TC><<<grid, kTcThreads, kTcSmem, st>>>(
      M, N, K, A, lda, B, ldb, C, ldc, kchunk, zstride, bias, relu ? 1 : 0, vec, status, g_loop_wait_limit);
  note_launches(1);
  return cudaGetLastError();
}

// C[m][n] = act(sum_z part[z][m][n] + bias[n]), the splits added in order.
__global__ void k_tc_sum(const float* __restrict__ part, int splits, int M, int N, float* __restrict__ C, int ldc,
                         const float* __restrict__ bias, int relu) {
  const long long MN = (long long)M * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * MN + i];
    const int n = (int)(i % N);
    if (bias) s += bias[n];
    if (relu) s = fmaxf(s, 0.f);
    C[(size_t)(i / N) * ldc + n] = s;
  }
}

}  // namespace

cudaError_t gemm_tc(bool at, bool bt, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                    int ldc, const float* bias, bool relu, int splits, long long zstride, int* status,
                    cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!at && !bt) return launch_tc<false, false>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, splits, zstride, status, st);
  if (!at && bt) return launch_tc<false, true>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, splits, zstride, status, st);
  if (at && !bt) return launch_tc<true, false>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, splits, zstride, status, st);
  return launch_tc<true, true>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, splits, zstride, status, st);
}

cudaError_t gemm_tc_sum(bool at, bool bt, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                        float* C, int ldc, const float* bias, bool relu, int splits, float* part, int* status,
                        cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splits <= 1) return gemm_tc(at, bt, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, 1, 0, status, st);
  cudaError_t e = gemm_tc(at, bt, M, N, K, A, lda, B, ldb, part, N, nullptr, false, splits, (long long)M * N, status, st);
  if (e != cudaSuccess) return e;
  const long long MN = (long long)M * N;
  k_tc_sum<<<(unsigned)std::min<long long>((MN + 255) / 256, 152LL * 16), 256, 0, st>>>(part, splits, M, N, C, ldc,
                                                                                     bias, relu ? 1 : 0);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs

extern "C" digs_status digs_set_wait_limit(long long tests) {
  digs::g_loop_wait_limit = tests < 0 ? digs::kWaitLimit : (unsigned)std::min<long long>(tests, 1LL << 30);
  return DIGS_OK;
}

extern "C" digs_status digs_gemm_bf16(int trans_a, int trans_b, int M, int N, int K, const float* A, int lda,
                                      const float* B, int ldb, const float* bias, int relu, float* C, int ldc,
                                      int splits, float* partial, int* status, void* stream) {
  using namespace digs;
  if (M < 0 || N < 0 || K < 0 || splits < 1 || splits > 64) return DIGS_ERR_ARG;
  if (M == 0 || N == 0) return DIGS_OK;
  if (!C || ldc < N || (K > 0 && (!A || !B))) return DIGS_ERR_ARG;
  if (K > 0 && (lda < (trans_a ? M : K) || ldb < (trans_b ? K : N))) return DIGS_ERR_ARG;
  if (splits > 1 && !partial) return DIGS_ERR_ARG;
  const cudaError_t e = gemm_tc_sum(trans_a != 0, trans_b != 0, M, N, K, A, lda, B, ldb, C, ldc, bias, relu != 0,
                                    splits, partial, status, (cudaStream_t)stream);
  return e == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}
