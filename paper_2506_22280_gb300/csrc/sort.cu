// Stable LSD radix sort of (projection, tile) keys with their slot values, 8 bits per pass, and the
// per-(projection, tile) ranges of the sorted list.  The pair count lives on the device (it comes out
// of the prefix sum), so every kernel is launched for the workspace capacity and reads the count.
//
// Each pass: (1) per-block digit histograms, stored digit-major; (2) an exclusive scan of that
// [256][blocks] array gives every (digit, block) its output base; (3) each block ranks its keys stably --
// each warp walks a contiguous run of 512 keys in order, ranking equal digits inside a 32-key step with
// __match_any_sync and across steps with per-warp digit counters -- and scatters them.
#include "digs_internal.h"

namespace digs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                               // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;         // 4096 keys per block
constexpr int kWarpRun = kSortTile / kSortWarps;             // 512 keys per warp

int sort_blocks(long long cap) { return (int)((cap + kSortTile - 1) / kSortTile); }

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys, const uint32_t* n_dev,
                                                             int shift, uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  uint32_t n = n_dev[1];
  size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int i = 0; i < kSortItems; ++i) {
    size_t idx = base + (size_t)i * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin,
                                                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                const uint32_t* n_dev, int shift,
                                                                const uint32_t* __restrict__ hist_scan, int nblk) {
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t dbase[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wcnt[w][threadIdx.x] = 0u;
  dbase[threadIdx.x] = hist_scan[(size_t)threadIdx.x * nblk + blockIdx.x];
  __syncthreads();
  const uint32_t n = n_dev[1];
  const size_t run = (size_t)blockIdx.x * kSortTile + (size_t)warp * kWarpRun;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    size_t idx = run + (size_t)it * 32 + lane;
    bool valid = idx < n;
    key[it] = valid ? kin[idx] : 0u;
    val[it] = valid ? vin[idx] : 0u;
    uint32_t d = valid ? ((key[it] >> shift) & 255u) : 256u;  // 256: sentinel for the ragged tail
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = __popc(peers & lt_mask);
    rank[it] = valid ? wcnt[warp][d] + before : 0u;
    __syncwarp();
    if (valid && before == 0) wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive scan of the per-warp counts of each digit, in warp order
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t c = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = acc;
      acc += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    size_t idx = run + (size_t)it * 32 + lane;
    if (idx < n) {
      uint32_t d = (key[it] >> shift) & 255u;
      uint32_t pos = dbase[d] + wcnt[warp][d] + rank[it];
      kout[pos] = key[it];
      vout[pos] = val[it];
    }
  }
}

cudaError_t radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, const uint32_t* n_dev,
                       long long cap, int bits, uint32_t* hist, uint32_t* scan_tmp, int nblk, uint32_t** out_keys,
                       uint32_t** out_vals, cudaStream_t st) {
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  if (cap > 0 && nblk > 0) {
    for (int shift = 0; shift < bits; shift += 8) {
      k_radix_hist<<<nblk, kSortThreads, 0, st>>>(ki, n_dev, shift, hist, nblk);
      cudaError_t e = exclusive_scan(hist, hist, 256 * nblk, scan_tmp, st);
      if (e != cudaSuccess) return e;
      k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(ki, vi, ko, vo, n_dev, shift, hist, nblk);
      note_launches(2);
      uint32_t* t = ki; ki = ko; ko = t;
      t = vi; vi = vo; vo = t;
    }
  }
  *out_keys = ki;
  *out_vals = vi;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ keys, const uint32_t* n_dev,
                                                     uint2* __restrict__ ranges) {
  uint32_t n = n_dev[1];
  size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  uint32_t key = keys[k];
  if (k == 0 || keys[k - 1] != key) ranges[key].x = (uint32_t)k;
  if (k + 1 == n || keys[k + 1] != key) ranges[key].y = (uint32_t)(k + 1);
}

cudaError_t tile_ranges(const uint32_t* sorted_keys, const uint32_t* n_dev, long long cap, uint2* ranges,
                        int n_ranges, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_ranges, st);
  if (e != cudaSuccess) return e;
  if (cap <= 0) return cudaSuccess;
  long long blocks = (cap + 255) / 256;
  k_tile_ranges<<<(unsigned)blocks, 256, 0, st>>>(sorted_keys, n_dev, ranges);
  note_launches(1);
  return cudaGetLastError();
}

// Launch order of the forward raster's CTAs: (projection, tile) indices by descending list length, in
// 33 power-of-two classes (longest first), so that the heaviest tiles start in the first wave and the
// tail of the launch is made of light ones.  Only the launch order depends on it, not any result.
__global__ void __launch_bounds__(1024) k_tile_order(const uint2* __restrict__ ranges, int n,
                                                     uint32_t* __restrict__ order) {
  __shared__ uint32_t cls[33];
  if (threadIdx.x < 33) cls[threadIdx.x] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint2 r = ranges[i];
    atomicAdd(&cls[__clz(r.y - r.x)], 1u);  // 0 for the longest lists, 32 for empty ones
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int c = 0; c < 33; ++c) {
      const uint32_t k = cls[c];
      cls[c] = acc;
      acc += k;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint2 r = ranges[i];
    order[atomicAdd(&cls[__clz(r.y - r.x)], 1u)] = (uint32_t)i;
  }
}

cudaError_t tile_order(const uint2* ranges, int n, uint32_t* order, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_tile_order<<<1, 1024, 0, st>>>(ranges, n, order);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs
