// Tile rasteriser of the X-ray transform (Sec. 3.1, Eq. 1, 3-4) and its backward pass.
//
// One CTA per (projection, tile).  The tile's (sorted) Gaussian list is staged into shared memory in
// chunks of 256 records with 16-byte vector loads; each warp then takes one Gaussian at a time and its
// lanes sweep the pixels of that Gaussian's box inside the tile.  The forward adds each pair's line
// integral into a per-warp tile accumulator (no atomics; warps merge in a fixed order at the end), so the
// result is deterministic.  The backward recomputes every pair, accumulates the ten sums that carry the
// record gradients in registers, reduces them across the warp with shuffles and writes them to the pair's
// slot; the per-Gaussian chain kernel then adds the slots of each Gaussian in order (again no atomics).
#include "digs_internal.h"

namespace digs {

constexpr int kRasterThreads = 256;
constexpr int kRasterWarps = kRasterThreads / 32;

struct PairEval {
  float dx, dy, num, t, D;
};

__device__ __forceinline__ bool eval_pair(const Rec& r, int px, int py, float c2, PairEval& p) {
  p.dx = (float)px - r.xc;
  p.dy = (float)py - r.yc;
  p.num = p.dx * fmaf(r.n00, p.dx, r.n01x2 * p.dy) + r.n11 * p.dy * p.dy;
  p.t = fmaf(r.wn0, p.dx, fmaf(r.wn1, p.dy, 1.f));
  p.D = fmaf(p.t, p.t, r.kappa * p.num);
  return p.num <= c2 * p.D;  // E = num / D <= c2, D > 0
}

template <int TS>
__global__ void __launch_bounds__(kRasterThreads) k_raster_fwd(
    const float4* __restrict__ rec, const uint32_t* __restrict__ svals, const uint32_t* __restrict__ rid,
    const uint2* __restrict__ ranges, const __grid_constant__ ViewsParam views, int tiles_x, int T, int nu, int nv,
    float c2, float* __restrict__ proj, const float* __restrict__ meas, float* __restrict__ dldi,
    float* __restrict__ loss_part, float inv_count, unsigned long long* __restrict__ counters) {
  constexpr int NPX = TS * TS;
  __shared__ float acc[kRasterWarps][NPX];
  __shared__ float4 srec[kRasterThreads * DIGS_REC_F4];
  __shared__ float red[kRasterWarps];
  const int b = blockIdx.y, tile = blockIdx.x;
  const int ox = (tile % tiles_x) * TS, oy = (tile / tiles_x) * TS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p = threadIdx.x; p < kRasterWarps * NPX; p += kRasterThreads) (&acc[0][0])[p] = 0.f;
  const uint2 rg = ranges[(size_t)b * T + tile];
  const ViewC& v = views.v[b];
  unsigned n_box = 0, n_cut = 0;  // per warp (lane 0) / per thread
  for (uint32_t base = rg.x; base < rg.y; base += kRasterThreads) {
    __syncthreads();
    uint32_t k = base + threadIdx.x;
    if (k < rg.y) {
      const float4* src = rec + (size_t)rid[svals[k]] * DIGS_REC_F4;
#pragma unroll
      for (int q = 0; q < DIGS_REC_F4; ++q) srec[threadIdx.x * DIGS_REC_F4 + q] = src[q];
    }
    __syncthreads();
    int cnt = min((int)(rg.y - base), kRasterThreads);
    for (int e = warp; e < cnt; e += kRasterWarps) {
      Rec r = load_rec(&srec[e * DIGS_REC_F4]);
      int x0 = max(r.bx & 0xffff, ox), x1 = min(r.bx >> 16, ox + TS - 1);
      int y0 = max(r.by & 0xffff, oy), y1 = min(r.by >> 16, oy + TS - 1);
      int wdt = x1 - x0 + 1, hgt = y1 - y0 + 1;
      if (wdt <= 0 || hgt <= 0) continue;  // cannot happen for keys emitted from the box; kept as a guard
      int npx = wdt * hgt;
      float inv_w = 1.f / (float)wdt;
      n_box += npx;
      for (int kk = lane; kk < npx; kk += 32) {
        int rr = (int)(((float)kk + 0.5f) * inv_w);
        int px = x0 + (kk - rr * wdt), py = y0 + rr;
        PairEval pe;
        if (eval_pair(r, px, py, c2, pe)) {
          float rs = rsqrtf(pe.D);
          float E = pe.num * rs * rs;
          acc[warp][(py - oy) * TS + (px - ox)] += r.amp * rs * exp2f(-0.5f * DIGS_LOG2E * E);
          ++n_cut;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  float lsum = 0.f;
  for (int p = threadIdx.x; p < NPX; p += kRasterThreads) {
    int px = ox + p % TS, py = oy + p / TS;
    if (px < nu && py < nv) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kRasterWarps; ++w) s += acc[w][p];
      float I = s * pixel_ray_length(v, (float)px, (float)py);
      size_t idx = ((size_t)b * nv + py) * nu + px;
      if (proj) proj[idx] = I;
      if (meas) {
        float res = I - meas[idx];
        lsum = fmaf(res, res, lsum);
        if (dldi) dldi[idx] = 2.f * res * inv_count;
      }
    }
  }
  if (counters) {
    unsigned c = n_cut;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && (n_box | c)) {
      atomicAdd(counters, (unsigned long long)n_box);
      atomicAdd(counters + 1, (unsigned long long)c);
    }
  }
  if (loss_part) {
    lsum = warp_sum(lsum);
    if (lane == 0) red[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < kRasterWarps; ++w) s += red[w];
      loss_part[(size_t)b * T + tile] = s;
    }
  }
}

template <int TS>
__global__ void __launch_bounds__(kRasterThreads) k_raster_bwd(
    const float4* __restrict__ rec, const uint32_t* __restrict__ svals, const uint32_t* __restrict__ rid,
    const uint2* __restrict__ ranges, const __grid_constant__ ViewsParam views, int tiles_x, int T, int nu, int nv,
    float c2, const float* __restrict__ grad_proj, float4* __restrict__ partials) {
  constexpr int NPX = TS * TS;
  __shared__ float gpix[NPX];
  __shared__ float4 srec[kRasterThreads * DIGS_REC_F4];
  __shared__ uint32_t sslot[kRasterThreads];
  const int b = blockIdx.y, tile = blockIdx.x;
  const int ox = (tile % tiles_x) * TS, oy = (tile / tiles_x) * TS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint2 rg = ranges[(size_t)b * T + tile];
  if (rg.x == rg.y) return;
  const ViewC& v = views.v[b];
  for (int p = threadIdx.x; p < NPX; p += kRasterThreads) {
    int px = ox + p % TS, py = oy + p / TS;
    float g = 0.f;
    if (px < nu && py < nv)
      g = grad_proj[((size_t)b * nv + py) * nu + px] * pixel_ray_length(v, (float)px, (float)py);
    gpix[p] = g;
  }
  for (uint32_t base = rg.x; base < rg.y; base += kRasterThreads) {
    __syncthreads();
    uint32_t k = base + threadIdx.x;
    if (k < rg.y) {
      uint32_t slot = svals[k];
      sslot[threadIdx.x] = slot;
      const float4* src = rec + (size_t)rid[slot] * DIGS_REC_F4;
#pragma unroll
      for (int q = 0; q < DIGS_REC_F4; ++q) srec[threadIdx.x * DIGS_REC_F4 + q] = src[q];
    }
    __syncthreads();
    int cnt = min((int)(rg.y - base), kRasterThreads);
    for (int e = warp; e < cnt; e += kRasterWarps) {
      Rec r = load_rec(&srec[e * DIGS_REC_F4]);
      int x0 = max(r.bx & 0xffff, ox), x1 = min(r.bx >> 16, ox + TS - 1);
      int y0 = max(r.by & 0xffff, oy), y1 = min(r.by >> 16, oy + TS - 1);
      int wdt = x1 - x0 + 1, hgt = y1 - y0 + 1;
      if (wdt <= 0 || hgt <= 0) continue;  // cannot happen for keys emitted from the box; kept as a guard
      int npx = wdt * hgt;
      float inv_w = 1.f / (float)wdt;
      float S[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) S[q] = 0.f;
      for (int kk = lane; kk < npx; kk += 32) {
        int rr = (int)(((float)kk + 0.5f) * inv_w);
        int px = x0 + (kk - rr * wdt), py = y0 + rr;
        PairEval pe;
        if (eval_pair(r, px, py, c2, pe)) {
          float g = gpix[(py - oy) * TS + (px - ox)];
          float rs = rsqrtf(pe.D);
          float inv_D = rs * rs;
          float E = pe.num * inv_D;
          float base_v = rs * exp2f(-0.5f * DIGS_LOG2E * E);  // V / amp
          float G = g * r.amp * base_v;                        // dL/dV * V
          float al = 0.5f * G * inv_D;
          float em1 = E - 1.f;
          float gnum = al * fmaf(r.kappa, em1, -1.f);
          float gt = 2.f * al * em1 * pe.t;
          float gnx = gnum * pe.dx, gny = gnum * pe.dy;
          S[0] = fmaf(g, base_v, S[0]);
          S[1] = fmaf(gnx, pe.dx, S[1]);
          S[2] = fmaf(gnx, pe.dy, S[2]);
          S[3] = fmaf(gny, pe.dy, S[3]);
          S[4] += gnx;
          S[5] += gny;
          S[6] += gt;
          S[7] = fmaf(gt, pe.dx, S[7]);
          S[8] = fmaf(gt, pe.dy, S[8]);
          S[9] = fmaf(al * em1, pe.num, S[9]);
        }
      }
#pragma unroll
      for (int q = 0; q < 10; ++q) S[q] = warp_sum(S[q]);
      if (lane == 0) {
        float4* dst = partials + (size_t)sslot[e] * DIGS_PARTIAL_F4;
        dst[0] = make_float4(S[0], S[1], S[2], S[3]);
        dst[1] = make_float4(S[4], S[5], S[6], S[7]);
        dst[2] = make_float4(S[8], S[9], 0.f, 0.f);
      }
    }
  }
}

cudaError_t launch_raster_fwd(const Workspace& ws, const uint32_t* sorted_vals, const ViewsParam& views, float c2,
                              float* proj, const float* meas, float* dldi, float inv_count, cudaStream_t st) {
  if (ws.P <= 0) return cudaSuccess;
  dim3 grid(ws.T, ws.P);
#define DIGS_RF(TS)                                                                                            \
  k_raster_fwd<TS><<<grid, kRasterThreads, 0, st>>>(ws.rec, sorted_vals, ws.rid, ws.ranges, views, ws.tiles_x,  \
                                                    ws.T, ws.nu, ws.nv, c2, proj, meas, dldi,                  \
                                                    meas ? ws.loss_part : nullptr, inv_count, ws.counters)
  switch (ws.tile) {
    case 8: DIGS_RF(8); break;
    case 16: DIGS_RF(16); break;
    case 32: DIGS_RF(32); break;
    default: return cudaErrorInvalidValue;
  }
#undef DIGS_RF
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const Workspace& ws, const uint32_t* sorted_vals, const ViewsParam& views, float c2,
                              const float* grad_proj, cudaStream_t st) {
  if (ws.P <= 0) return cudaSuccess;
  dim3 grid(ws.T, ws.P);
#define DIGS_RB(TS)                                                                                           \
  k_raster_bwd<TS><<<grid, kRasterThreads, 0, st>>>(ws.rec, sorted_vals, ws.rid, ws.ranges, views, ws.tiles_x, \
                                                    ws.T, ws.nu, ws.nv, c2, grad_proj, ws.partials)
  switch (ws.tile) {
    case 8: DIGS_RB(8); break;
    case 16: DIGS_RB(16); break;
    case 32: DIGS_RB(32); break;
    default: return cudaErrorInvalidValue;
  }
#undef DIGS_RB
  note_launches(1);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_loss_reduce(const float* __restrict__ part, int n, float* out,
                                                      float scale) {
  __shared__ float red[32];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[0] = t * scale;
  }
}

cudaError_t launch_loss_reduce(const float* part, int n, float* out, float scale, cudaStream_t st) {
  // part holds per-tile sums of squared residuals; out[0] = scale * their sum
  k_loss_reduce<<<1, 1024, 0, st>>>(part, n, out, scale);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs
