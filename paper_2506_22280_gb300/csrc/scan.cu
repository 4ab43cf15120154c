// Device-wide exclusive prefix sum of uint32 counts (three passes: block sums, scan of block sums,
// block-local scan plus block offset).  out has n + 1 entries; out[n] is the total.
#include "digs_internal.h"

namespace digs {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_words(int n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 2; }

// Exclusive scan of one value per thread across the block; returns the block total in *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tot, uint32_t* total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    uint32_t t = lane < nw ? warp_tot[lane] : 0u;
    uint32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_tot[lane] = s - t;  // exclusive warp offsets
    if (lane == 31) *total = s;
  }
  __syncthreads();
  uint32_t r = warp_tot[warp] + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, int n,
                                                              uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t total;
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < (size_t)n) s += in[base + i];
  block_excl_scan(s, warp_tot, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t* __restrict__ block_sums, int nb) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t total;
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += kScanThreads) {
    int i = base + threadIdx.x;
    uint32_t v = i < nb ? block_sums[i] : 0u;
    uint32_t e = block_excl_scan(v, warp_tot, &total);
    if (i < nb) block_sums[i] = carry + e;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                             int n, const uint32_t* __restrict__ block_sums, int nb) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t total;
  size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < (size_t)n ? in[base + i] : 0u;
    s += v[i];
  }
  uint32_t e = block_excl_scan(s, warp_tot, &total) + block_sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < (size_t)n) out[base + i] = e;
    e += v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = block_sums[nb];
}

__global__ void k_scan_empty(uint32_t* out) { out[0] = 0u; }

cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int n, uint32_t* tmp, cudaStream_t st) {
  if (n <= 0) {
    k_scan_empty<<<1, 1, 0, st>>>(out);
    note_launches(1);
    return cudaGetLastError();
  }
  int nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, tmp);
  k_scan_top<<<1, kScanThreads, 0, st>>>(tmp, nb);
  k_scan_apply<<<nb, kScanThreads, 0, st>>>(in, out, n, tmp, nb);
  note_launches(3);
  return cudaGetLastError();
}

}  // namespace digs
