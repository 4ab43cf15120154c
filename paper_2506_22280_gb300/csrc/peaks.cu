// Microbenchmarks of the arithmetic pipes the splat kernels are bound by: the FP32 FMA pipe (scalar
// fma.rn.f32 and packed fma.rn.f32x2) and the SFU (ex2.approx and rsqrt.approx, the two special
// functions of every (pixel, Gaussian) pair).  The caller times a launch with CUDA events on its stream
// and divides the lane operations the launch performs by that time; the measured rates are the peaks
// the roofline fractions of the raster kernels are taken against.
//
// Every thread runs eight independent dependency chains for `iters` iterations (enough independent
// work per warp that issue, not latency, limits a full SM); the grid is two CTAs of 1024 threads per SM.
// A lane operation is one FP32 result: an FMA counts once, a packed FMA twice, an SFU result once.
#include "digs_internal.h"

namespace digs {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 1024;

__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// kind 0: scalar FMA chains x = x * a + b; kind 1: the same in packed pairs; kind 2: x = 2^-x;
// kind 3: x = 1 / sqrt(x).  The chains stay finite and away from denormals: the FMA chains converge
// to b / (1 - a), 2^-x stays in [0.5, 1], 1/sqrt(x) tends to 1.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_pipe(int iters, float seed, float* __restrict__ sink) {
  const float s = seed + 1e-3f * (float)(threadIdx.x & 7);
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = s + 0.01f * (float)c;
  if (KIND == 0) {
    const float a = 0.999f, b = 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
  } else if (KIND == 1) {
    unsigned long long v[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) v[c] = pk2(x[2 * c], x[2 * c + 1]);
    const unsigned long long a = pk2(0.999f, 0.999f), b = pk2(1e-3f, 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[c]) : "l"(a), "l"(b));
    }
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) upk2(v[c], x[2 * c], x[2 * c + 1]);
  } else if (KIND == 2) {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(-x[c]));
    }
  } else {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
    }
  }
  float t = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += x[c];
  if (t == -1.f) sink[0] = t;  // never true; keeps the chains live
}

}  // namespace
}  // namespace digs

extern "C" digs_status digs_pipe_bench(int kind, int iters, float* sink, long long* lane_ops, void* stream) {
  using namespace digs;
  if (kind < 0 || kind > 3 || iters < 1 || !sink || !lane_ops) return DIGS_ERR_ARG;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DIGS_ERR_CUDA;
  const dim3 grid(2 * n_sm);
  cudaStream_t st = (cudaStream_t)stream;
  switch (kind) {
    case 0: k_pipe<0><<<grid, kPeakThreads, 0, st>>>(iters, 0.5f, sink); break;
    case 1: k_pipe<1><<<grid, kPeakThreads, 0, st>>>(iters, 0.5f, sink); break;
    case 2: k_pipe<2><<<grid, kPeakThreads, 0, st>>>(iters, 0.5f, sink); break;
    default: k_pipe<3><<<grid, kPeakThreads, 0, st>>>(iters, 0.5f, sink); break;
  }
  note_launches(1);
  // per thread and iteration: 4 x 8 scalar results (kinds 0, 2, 3) or 8 x 4 packed pairs, 64 results (kind 1)
  *lane_ops = (long long)grid.x * kPeakThreads * (long long)iters * (kind == 1 ? 64LL : 32LL);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}
