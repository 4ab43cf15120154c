// Binning of the (projection, tile) pairs into per-tile record lists.  Up to kDirectMaxTiles tiles per
// projection, bin_direct (below) counts and places the pairs straight from the records' tile rectangles.
// Beyond that, sort_pairs: a stable sort of the emitted (projection, tile) pair keys with their record
// values, and the per-(projection, tile) ranges of the sorted list.  The pairs come out of the emit step
// projection by projection, so
// only the tile part of each key needs sorting, inside each projection's run: an LSD radix sort on the
// tile index, 8 bits per pass (one pass when a projection has at most 256 tiles), whose blocks never
// straddle two projections.  The pair count lives on the device (it comes out of the prefix sum), so
// every kernel is launched for the workspace capacity and reads the counts.
//
// Each pass: (1) per-block digit histograms, stored projection-major, then digit-major, then by block,
// so that (2) one exclusive scan of the whole array gives every (projection, digit, block) its output
// base; (3) each block ranks its keys stably -- each warp walks a contiguous run of 512 keys in order,
// ranking equal digits inside a 32-key step with __match_any_sync and across steps with per-warp digit
// counters -- puts them in sorted order in shared memory and writes each digit's run out contiguously.
// With one pass the ranges follow from the scanned histograms.
#include "digs_internal.h"

namespace digs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                               // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;         // 4096 keys per block
constexpr int kWarpRun = kSortTile / kSortWarps;             // 512 keys per warp

// Upper bound of the sort blocks: every projection's run may end in a partial block.
int sort_blocks(long long cap, int P) { return (int)((cap + kSortTile - 1) / kSortTile) + P; }

// seg[0..P]: start of each projection's pairs (seg[P] = pairs kept); seg[P+1..2P+1]: first sort block of
// each projection (seg[2P+1] = blocks in use).  One CTA of 256 threads, P <= 255.
__global__ void __launch_bounds__(256) k_sort_segments(const uint32_t* __restrict__ offsets,
                                                       const uint32_t* __restrict__ n_dev, int n, int P,
                                                       uint32_t* __restrict__ seg) {
  __shared__ uint32_t start[257], nb[256];
  const int t = threadIdx.x;
  const uint32_t kept = n_dev[1];
  if (t <= P) start[t] = t < P ? min(offsets[(size_t)t * n], kept) : kept;
  __syncthreads();
  uint32_t x = t < P ? (start[t + 1] - start[t] + kSortTile - 1) / kSortTile : 0u;
  nb[t] = x;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {  // inclusive scan of the block counts
    const uint32_t y = t >= o ? nb[t - o] : 0u;
    __syncthreads();
    x += y;
    nb[t] = x;
    __syncthreads();
  }
  if (t <= P) {
    seg[t] = start[t];
    seg[P + 1 + t] = t == 0 ? 0u : nb[t - 1];
  }
}

// The projection whose sort blocks hold block g (the last b with first block <= g; g < blocks in use).
__device__ __forceinline__ int block_projection(const uint32_t* sblk, int P, uint32_t g) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sblk[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct SortBlock {
  bool idle;
  int b;            // projection
  uint32_t j, nb;   // block within the projection, blocks of the projection
  uint32_t lo, hi;  // keys [lo, hi)
  uint32_t hbase;   // first histogram entry of the projection
};

__device__ __forceinline__ SortBlock sort_block(const uint32_t* seg, int P) {
  const uint32_t* sblk = seg + P + 1;
  SortBlock s;
  const uint32_t g = blockIdx.x;
  s.idle = g >= sblk[P];
  if (s.idle) return s;
  s.b = block_projection(sblk, P, g);
  s.j = g - sblk[s.b];
  s.nb = sblk[s.b + 1] - sblk[s.b];
  s.lo = seg[s.b] + s.j * kSortTile;
  s.hi = min(s.lo + (uint32_t)kSortTile, seg[s.b + 1]);
  s.hbase = 256u * sblk[s.b];
  return s;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ seg, int P, int T, int shift,
                                                            uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  const SortBlock s = sort_block(seg, P);
  if (s.idle) {  // idle blocks zero the tail of the histogram array, which the scan covers
    hist[(size_t)blockIdx.x * 256 + threadIdx.x] = 0u;
    return;
  }
  h[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t kb = (uint32_t)s.b * (uint32_t)T;
  uint32_t k[kSortItems];  // every load issued before the first use
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = s.lo + (uint32_t)(i * kSortThreads) + threadIdx.x;
    k[i] = idx < s.hi ? keys[idx] : 0u;
  }
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = s.lo + (uint32_t)(i * kSortThreads) + threadIdx.x;
    if (idx < s.hi) atomicAdd(&h[((k[i] - kb) >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[s.hbase + threadIdx.x * s.nb + s.j] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads, 3) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               const uint32_t* __restrict__ seg, int P, int T, int shift,
                                                               const uint32_t* __restrict__ hist_scan) {
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t dbase[256];   // output position of the block's first key of each digit
  __shared__ uint32_t loff[256];    // position of that key inside the block's sorted run
  __shared__ uint32_t wsum[kSortWarps];
  __shared__ uint32_t sk[kSortTile], sv[kSortTile];
  const SortBlock s = sort_block(seg, P);
  if (s.idle) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wcnt[w][threadIdx.x] = 0u;
  dbase[threadIdx.x] = hist_scan[s.hbase + threadIdx.x * s.nb + s.j];
  __syncthreads();
  const uint32_t kb = (uint32_t)s.b * (uint32_t)T;
  const uint32_t run = s.lo + (uint32_t)(warp * kWarpRun);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {  // every load issued before the ranking needs the first
    const uint32_t idx = run + (uint32_t)(it * 32 + lane);
    const bool valid = idx < s.hi;
    key[it] = valid ? kin[idx] : 0u;
    val[it] = valid ? vin[idx] : 0u;
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const uint32_t idx = run + (uint32_t)(it * 32 + lane);
    const bool valid = idx < s.hi;
    const uint32_t d = valid ? (((key[it] - kb) >> shift) & 255u) : 256u;  // 256: sentinel for the ragged tail
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt_mask);
    rank[it] = valid ? wcnt[warp][d] + before : 0u;
    __syncwarp();
    if (valid && before == 0) wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  uint32_t total = 0;  // keys of digit threadIdx.x in the block
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {  // exclusive scan of the per-warp counts of each digit, in warp order
    const uint32_t c = wcnt[w][threadIdx.x];
    wcnt[w][threadIdx.x] = total;
    total += c;
  }
  {  // exclusive scan of the digit totals over the digits: each digit's run inside the block
    uint32_t x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before_w = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) before_w += w < warp ? wsum[w] : 0u;
    loff[threadIdx.x] = before_w + x - total;
  }
  __syncthreads();
  // the block's keys in sorted order in shared memory, then written out run by run (coalesced)
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const uint32_t idx = run + (uint32_t)(it * 32 + lane);
    if (idx < s.hi) {
      const uint32_t d = ((key[it] - kb) >> shift) & 255u;
      const uint32_t p = loff[d] + wcnt[warp][d] + rank[it];
      sk[p] = key[it];
      sv[p] = val[it];
    }
  }
  __syncthreads();
  const uint32_t cnt = s.hi - s.lo;
  for (uint32_t i = threadIdx.x; i < cnt; i += kSortThreads) {
    const uint32_t k = sk[i];
    const uint32_t d = ((k - kb) >> shift) & 255u;
    const uint32_t pos = dbase[d] + (i - loff[d]);
    if (kout) kout[pos] = k;
    vout[pos] = sv[i];
  }
}

// With one pass (T <= 256) the digit is the tile, so the scanned histogram entry of (projection, tile,
// first block) is where the tile's run starts.
__global__ void __launch_bounds__(256) k_sort_ranges(const uint32_t* __restrict__ hist_scan,
                                                     const uint32_t* __restrict__ seg, int P, int T,
                                                     uint2* __restrict__ ranges) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * T) return;
  const int b = i / T, t = i - b * T;
  const uint32_t* sblk = seg + P + 1;
  const uint32_t nb = sblk[b + 1] - sblk[b], hb = 256u * sblk[b];
  uint2 r;
  if (nb == 0) {
    r.x = r.y = seg[b];
  } else {
    r.x = hist_scan[hb + (uint32_t)t * nb];
    r.y = t + 1 < 256 ? hist_scan[hb + (uint32_t)(t + 1) * nb] : seg[b + 1];
  }
  ranges[i] = r;
}

cudaError_t sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, const uint32_t* n_dev,
                       long long cap, const uint32_t* offsets, int n, int P, int T, int n_blocks, uint32_t* seg,
                       uint32_t* hist,
                       uint32_t* scan_tmp, uint2* ranges, uint32_t** out_keys, uint32_t** out_vals, cudaStream_t st) {
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  *out_keys = ki;
  *out_vals = vi;
  if (P <= 0 || T <= 0) return cudaSuccess;
  if (P > 255) return cudaErrorInvalidValue;
  int bits = 1;
  while ((1 << bits) < T) ++bits;
  k_sort_segments<<<1, 256, 0, st>>>(offsets, n_dev, n, P, seg);
  note_launches(1);
  for (int shift = 0; shift < bits; shift += 8) {
    k_sort_hist<<<n_blocks, kSortThreads, 0, st>>>(ki, seg, P, T, shift, hist);
    cudaError_t e = exclusive_scan(hist, hist, 256 * n_blocks, scan_tmp, st);
    if (e != cudaSuccess) return e;
    // with one pass the sorted keys are not needed (the ranges come from the scanned histogram)
    k_sort_scatter<<<n_blocks, kSortThreads, 0, st>>>(ki, vi, bits > 8 ? ko : nullptr, vo, seg, P, T, shift, hist);
    note_launches(2);
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  *out_keys = bits > 8 ? ki : nullptr;
  *out_vals = vi;
  if (bits <= 8) {
    k_sort_ranges<<<(P * T + 255) / 256, 256, 0, st>>>(hist, seg, P, T, ranges);
    note_launches(1);
    return cudaGetLastError();
  }
  return tile_ranges(ki, n_dev, cap, ranges, P * T, st);
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

// ---- direct binning: a counting sort of the (projection, tile) pairs, for T <= kDirectMaxTiles ----
// The records of a projection are cut into chunks of kBinChunk; k_bin_count counts each chunk's pairs per
// tile, a scan over (projection, tile, chunk) turns the counts into positions, and k_bin_scatter writes
// every pair's record id at its position: tile lists hold their records by chunk, then warp, then the
// pair's place in its record's tile rectangle (row-major), then lane -- a fixed order, so the forward's
// sums stay deterministic.  No keys are written and nothing is sorted.
constexpr int kBinChunk = 256;
constexpr int kBinWarps = kBinChunk / 32;

int bin_chunks(int n, int T) { return T <= kDirectMaxTiles ? (n + kBinChunk - 1) / kBinChunk : -1; }

__device__ __forceinline__ void unpack_tbox(uint2 v, int& tx0, int& ty0, int& tx1, int& ty1) {
  tx0 = (int)(v.x & 0xffffu); ty0 = (int)(v.x >> 16); tx1 = (int)(v.y & 0xffffu); ty1 = (int)(v.y >> 16);
}

// Grid (chunks, P): chist[(b T + t) C + c] = pairs of tile t among chunk c's records of projection b.
__global__ void __launch_bounds__(kBinChunk) k_bin_count(const uint2* __restrict__ tbox,
                                                         const uint32_t* __restrict__ counts, int N, int T,
                                                         int tiles_x, int C, uint32_t* __restrict__ chist) {
  __shared__ uint32_t h[kDirectMaxTiles];
  const int c = blockIdx.x, b = blockIdx.y;
  for (int t = threadIdx.x; t < T; t += kBinChunk) h[t] = 0u;
  __syncthreads();
  const int n = c * kBinChunk + threadIdx.x;
  if (n < N) {
    const size_t i = (size_t)b * N + n;
    if (counts[i] != 0u) {
      int tx0, ty0, tx1, ty1;
      unpack_tbox(tbox[i], tx0, ty0, tx1, ty1);
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&h[ty * tiles_x + tx], 1u);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += kBinChunk) chist[((size_t)b * T + t) * C + c] = h[t];
}

// Grid (chunks, P): every pair's record id b N + n at its position (cscan: the scanned chist).  Pairs at
// or past cap are dropped (k_bin_ranges flags them).
__global__ void __launch_bounds__(kBinChunk) k_bin_scatter(const uint2* __restrict__ tbox,
                                                           const uint32_t* __restrict__ counts, int N, int T,
                                                           int tiles_x, int C, const uint32_t* __restrict__ cscan,
                                                           long long cap, uint32_t* __restrict__ srid) {
  __shared__ uint32_t wpos[kBinWarps * kDirectMaxTiles];  // per warp and tile: pairs, then next position
  const int c = blockIdx.x, b = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = threadIdx.x; o < kBinWarps * T; o += kBinChunk) wpos[o] = 0u;
  __syncthreads();
  const int n = c * kBinChunk + threadIdx.x;
  int cnt = 0, tx0 = 0, ty0 = 0, tx1 = 0, wt = 1;
  if (n < N) {
    const size_t i = (size_t)b * N + n;
    if (counts[i] != 0u) {
      int ty1;
      unpack_tbox(tbox[i], tx0, ty0, tx1, ty1);
      wt = tx1 - tx0 + 1;
      cnt = wt * (ty1 - ty0 + 1);
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&wpos[warp * T + ty * tiles_x + tx], 1u);
    }
  }
  __syncthreads();
  // each tile's first position for each warp: the chunk's base plus the pairs of the earlier warps
  for (int t = threadIdx.x; t < T; t += kBinChunk) {
    uint32_t run = cscan[((size_t)b * T + t) * C + c];
#pragma unroll
    for (int w = 0; w < kBinWarps; ++w) {
      const uint32_t x = wpos[w * T + t];
      wpos[w * T + t] = run;
      run += x;
    }
  }
  __syncthreads();
  // the warp's pairs, slot k of every lane's rectangle at a time, lanes in order within a tile
  const int kmax = __reduce_max_sync(0xffffffffu, cnt);
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t rid = (uint32_t)((size_t)b * N + n);
  int cx = tx0, ct = ty0 * tiles_x + tx0;  // slot k's tile column and index, stepped row-major
  for (int k = 0; k < kmax; ++k) {
    const bool has = k < cnt;
    const int t = has ? ct : T;  // T: no pair in this slot
    if (++cx > tx1) {
      cx = tx0;
      ct += tiles_x - wt + 1;
    } else {
      ++ct;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    if (has) {
      const uint32_t pos = wpos[warp * T + t] + (uint32_t)__popc(peers & lt);
      if ((long long)pos < cap) srid[pos] = rid;
    }
    __syncwarp();
    if (has && (peers & lt) == 0u) wpos[warp * T + t] += (uint32_t)__popc(peers);
    __syncwarp();
  }
}

// ranges[j] of the PT (projection, tile) lists from the scan (clamped to cap); the pair counts and the
// capacity flag.
__global__ void __launch_bounds__(256) k_bin_ranges(const uint32_t* __restrict__ cscan, int PT, int C,
                                                    long long cap, uint2* __restrict__ ranges,
                                                    uint32_t* __restrict__ n_pairs, int* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t total = cscan[(size_t)PT * C];
  if (j == 0) {
    n_pairs[0] = total;
    n_pairs[1] = (long long)total > cap ? (uint32_t)cap : total;
    if ((long long)total > cap) set_status(status, DIGS_ERR_CAPACITY);
  }
  if (j >= PT) return;
  const long long x = cscan[(size_t)j * C], y = cscan[(size_t)(j + 1) * C];
  ranges[j] = make_uint2((uint32_t)(x < cap ? x : cap), (uint32_t)(y < cap ? y : cap));
}

cudaError_t bin_direct(const Workspace& ws, cudaStream_t st) {
  const int C = ws.n_chunks, PT = ws.P * ws.T;
  if (C > 0) {
    k_bin_count<<<dim3(C, ws.P), kBinChunk, 0, st>>>(ws.tbox, ws.counts, ws.n, ws.T, ws.tiles_x, C, ws.chist);
    note_launches(1);
  }
  cudaError_t e = exclusive_scan(ws.chist, ws.chist, PT * C, ws.scan_tmp, st);
  if (e != cudaSuccess) return e;
  if (C > 0) {
    k_bin_scatter<<<dim3(C, ws.P), kBinChunk, 0, st>>>(ws.tbox, ws.counts, ws.n, ws.T, ws.tiles_x, C, ws.chist,
                                                       ws.cap, ws.vals);
    note_launches(1);
  }
  if (PT > 0) {
    k_bin_ranges<<<(PT + 255) / 256, 256, 0, st>>>(ws.chist, PT, C, ws.cap, ws.ranges, ws.n_pairs, ws.status);
    note_launches(1);
  }
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
