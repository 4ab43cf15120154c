// Per-Gaussian forward preparation: FFD evaluation (Sec. 3.3, Eq. 10-11), deformation-informed warp of
// mean and covariance for every projection of the call (Sec. 3.2, Eq. 7-8), projection records with
// their pixel boxes, and emission of one (projection, tile) key per tile a box touches.
#include "digs_internal.h"
#include "ffd.cuh"
#include "setup.cuh"

namespace digs {

template <int R>
__global__ void __launch_bounds__(128) k_ffd_eval(LatticeC L, const float* __restrict__ phi,
                                                  const float* __restrict__ x, int n, float* __restrict__ U,
                                                  float* __restrict__ dU) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  float u[R][3], du[R][9];
  ffd_eval_point<R>(phi, L, p, u, du);
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) U[((size_t)i * R + r) * 3 + c] = u[r][c];
#pragma unroll
    for (int c = 0; c < 9; ++c) dU[((size_t)i * R + r) * 9 + c] = du[r][c];
  }
}

cudaError_t launch_ffd_eval(const LatticeC& L, const float* phi, const float* x, int n, float* U, float* dU,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid((n + 127) / 128);
  switch (L.R) {
    case 1: k_ffd_eval<1><<<grid, 128, 0, st>>>(L, phi, x, n, U, dU); break;
    case 2: k_ffd_eval<2><<<grid, 128, 0, st>>>(L, phi, x, n, U, dU); break;
    case 3: k_ffd_eval<3><<<grid, 128, 0, st>>>(L, phi, x, n, U, dU); break;
    case 4: k_ffd_eval<4><<<grid, 128, 0, st>>>(L, phi, x, n, U, dU); break;
    default: return cudaErrorInvalidValue;
  }
  note_launches(1);
  return cudaGetLastError();
}

// Reference Gaussian in registers: normalised quaternion, rotation, inverse scales.
struct GaussLocal {
  float mu0[3], s[3], inv_s[3], qh[4], qnorm, R[9], rho;
};

__device__ __forceinline__ void load_gauss(const GaussPtrs& g, int n, GaussLocal& o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o.mu0[c] = g.mu0[3 * n + c];
    o.s[c] = g.scale[3 * n + c];
    o.inv_s[c] = 1.f / o.s[c];
  }
  float q[4] = {g.quat[4 * n], g.quat[4 * n + 1], g.quat[4 * n + 2], g.quat[4 * n + 3]};
  o.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  float iq = 1.f / o.qnorm;
#pragma unroll
  for (int c = 0; c < 4; ++c) o.qh[c] = q[c] * iq;
  quat_to_R(o.qh, o.R);
  o.rho = g.rho[n];
}

// (1) One thread per Gaussian: u_r and grad u_r at its reference mean (the FFD, Eq. 10-11), kept for the
// set-up and the backward in component-major order ([12 R][n]: coalesced for every pass that reads them).
template <int R>
__global__ void __launch_bounds__(128) k_prep_ffd(GaussPtrs g, const __grid_constant__ ScanTable sc, LatticeC L,
                                                  const float* __restrict__ phi, float* __restrict__ ffd_out) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= g.n) return;
  const int s = scan_of(sc, gi);
  const float x[3] = {g.mu0[3 * gi], g.mu0[3 * gi + 1], g.mu0[3 * gi + 2]};
  float U[R][3], dU[R][9];
  ffd_eval_point<R>(phi + s * sc.phi_stride, L, x, U, dU);
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) ffd_out[(size_t)(r * 3 + c) * g.n + gi] = U[r][c];
#pragma unroll
    for (int c = 0; c < 9; ++c) ffd_out[(size_t)(3 * R + r * 9 + c) * g.n + gi] = dU[r][c];
  }
}

// (2) One thread per (Gaussian, group of kPrepGroup projections): the deformation-informed warp (Eq. 7-8)
// and the projection record of each projection of the group that renders the Gaussian's scan.
// Record (b, n) of scan-local Gaussian n sits at b * nmax + n.  Grid: (ceil(n / 128), ceil(P / kPrepGroup)).
constexpr int kPrepGroup = 16;
template <int R>
__global__ void __launch_bounds__(128, 5) k_prep_fwd(GaussPtrs g, const __grid_constant__ ScanTable sc,
                                                  const float* __restrict__ w, const __grid_constant__ ViewsParam views,
                                                  int P, float c2, int tile, float4* __restrict__ rec,
                                                  uint32_t* __restrict__ counts, uint2* __restrict__ tbox,
                                                  uint8_t* __restrict__ bcost, const float* __restrict__ ffd,
                                                  int* status) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= g.n) return;
  const int s = scan_of(sc, gi), n = gi - sc.off[s];
  GaussLocal G;
  load_gauss(g, gi, G);
  float U[R][3], dU[R][9];
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) U[r][c] = ffd[(size_t)(r * 3 + c) * g.n + gi];
#pragma unroll
    for (int c = 0; c < 9; ++c) dU[r][c] = ffd[(size_t)(3 * R + r * 9 + c) * g.n + gi];
  }
  const bool finite_in = isfinite(G.mu0[0] + G.mu0[1] + G.mu0[2] + G.s[0] + G.s[1] + G.s[2] + G.qnorm + G.rho);
  if (!finite_in && blockIdx.y == 0) set_status(status, DIGS_ERR_NONFINITE);
  const int b1 = min(P, ((int)blockIdx.y + 1) * kPrepGroup);
  for (int b = (int)blockIdx.y * kPrepGroup; b < b1; ++b) {
    const ViewC& v = views.v[b];
    if (v.scan != s) continue;
    const float* wb = w + (size_t)v.w_row * R;
    float mu[3], K[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) mu[c] = G.mu0[c];
#pragma unroll
    for (int c = 0; c < 9; ++c) K[c] = (c % 4 == 0) ? 1.f : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float wr = __ldg(wb + r);
#pragma unroll
      for (int c = 0; c < 3; ++c) mu[c] = fmaf(wr, U[r][c], mu[c]);
#pragma unroll
      for (int c = 0; c < 9; ++c) K[c] = fmaf(wr, dU[r][c], K[c]);
    }
    float Ki[9], A[9];
    float detK = inv3(K, Ki);
    Rec r;
    uint32_t cnt = 0, cost = 0;
    uint2 tb = make_uint2(0u, 0u);
    bool alive = finite_in && detK > DIGS_FOLD_EPS;
    if (alive) {
      make_A(G.inv_s, G.R, Ki, A);
      alive = v.ewa ? ewa_record(v, mu, A, G.rho, c2, r) : setup_record(v, mu, A, G.rho, c2, r);
    }
    if (alive) {
      int x0 = r.bx & 0xffff, x1 = r.bx >> 16, y0 = r.by & 0xffff, y1 = r.by >> 16;
      cnt = (uint32_t)((x1 / tile - x0 / tile + 1) * (y1 / tile - y0 / tile + 1));
      tb = make_uint2((uint32_t)(x0 / tile) | ((uint32_t)(y0 / tile) << 16), (uint32_t)(x1 / tile) | ((uint32_t)(y1 / tile) << 16));
      cost = min(((uint32_t)(x1 - x0 + 1) * (uint32_t)(y1 - y0 + 1) + 31u) >> 5, 255u);  // backward passes
    } else {
      r = Rec{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0, 0, 0};
    }
    size_t idx = (size_t)b * sc.nmax + n;
    store_rec(rec + idx * DIGS_REC_F4, r);
    counts[idx] = cnt;
    tbox[idx] = tb;
    bcost[idx] = (uint8_t)cost;
  }
}

cudaError_t launch_prep_fwd(const GaussPtrs& g, const ScanTable& sc, const LatticeC& L, const float* phi,
                            const float* w, const ViewsParam& views, int P, float c2, const Workspace& ws,
                            cudaStream_t st) {
  if (g.n <= 0 || P <= 0) return cudaSuccess;
  if (sc.S > 1) {  // records of projections whose scan is smaller than nmax are padding: no tiles
    cudaError_t e = cudaMemsetAsync(ws.counts, 0, (size_t)P * sc.nmax * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.n + 127) / 128);
  dim3 grid2(grid.x, (P + kPrepGroup - 1) / kPrepGroup);
#define DIGS_PREP(RR)                                                                                        \
  k_prep_ffd<RR><<<grid, 128, 0, st>>>(g, sc, L, phi, ws.ffd);                                                \
  k_prep_fwd<RR><<<grid2, 128, 0, st>>>(g, sc, w, views, P, c2, ws.tile, ws.rec, ws.counts, ws.tbox, ws.bcost, \
                                        ws.ffd, ws.status)
  switch (L.R) {
    case 1: DIGS_PREP(1); break;
    case 2: DIGS_PREP(2); break;
    case 3: DIGS_PREP(3); break;
    case 4: DIGS_PREP(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef DIGS_PREP
  note_launches(2);
  return cudaGetLastError();
}

// Each warp emits the pairs of 32 consecutive (projection, Gaussian) records i: key = b * T + tile and
// value i for each tile of i's box (rows of tiles, then tiles within a row), at the slots
// [offsets[i], offsets[i + 1]) reserved by the scan, so that after the stable sort the values are the
// record of each sorted position.  The warp's slots form one contiguous range; its lanes walk it 32 at a
// time (coalesced stores), each finding the record that owns its slot by a binary search over the
// warp's 32 offsets.  Pairs beyond the capacity are dropped and flagged.
__global__ void __launch_bounds__(256) k_emit(const float4* __restrict__ rec, const uint32_t* __restrict__ offsets,
                                              int PN, int n, int tile, int tiles_x, int T, uint32_t* __restrict__ keys,
                                              uint32_t* __restrict__ vals, long long cap, uint32_t* n_pairs,
                                              int* status) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt == 0) {
    const uint32_t total = offsets[PN];
    n_pairs[0] = total;
    n_pairs[1] = (long long)total > cap ? (uint32_t)cap : total;
    if ((long long)total > cap) set_status(status, DIGS_ERR_CAPACITY);
  }
  const int lane = threadIdx.x & 31;
  const int i0 = gt - lane;  // the warp's first record
  if (i0 >= PN) return;      // whole warps only
  const int i = i0 + lane;
  const uint32_t off = i < PN ? offsets[i] : offsets[PN];
  const uint32_t base = __shfl_sync(0xffffffffu, off, 0);
  const uint32_t last = offsets[min(i0 + 32, PN)];
  int tx0 = 0, w = 1, ty0 = 0;
  if (i < PN && offsets[i + 1] != off) {
    const float4 c = rec[(size_t)i * DIGS_REC_F4 + 2];
    const int bx = __float_as_int(c.y), by = __float_as_int(c.z);
    tx0 = (bx & 0xffff) / tile;
    ty0 = (by & 0xffff) / tile;
    w = (bx >> 16) / tile - tx0 + 1;
  }
  for (uint32_t k0 = base; k0 < last; k0 += 32) {  // the same trip count on every lane (shuffles below)
    const uint32_t k = k0 + lane;
    int r = 0;  // the last lane whose first slot is <= k (records with no slots share their successor's)
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t o = __shfl_sync(0xffffffffu, off, r + step);
      if (o <= k) r += step;
    }
    const uint32_t t = k - __shfl_sync(0xffffffffu, off, r);
    const int rw = __shfl_sync(0xffffffffu, w, r), rx0 = __shfl_sync(0xffffffffu, tx0, r);
    const int ry0 = __shfl_sync(0xffffffffu, ty0, r);
    const int ty = ry0 + (int)(t / (uint32_t)rw), tx = rx0 + (int)(t % (uint32_t)rw);
    if (k < last && (long long)k < cap) {
      const int ri = i0 + r;
      keys[k] = (uint32_t)(ri / n) * (uint32_t)T + (uint32_t)(ty * tiles_x + tx);
      vals[k] = (uint32_t)ri;
    }
  }
}

cudaError_t launch_emit(const Workspace& ws, cudaStream_t st) {
  int PN = ws.P * ws.n;
  dim3 grid((PN + 255) / 256 > 0 ? (PN + 255) / 256 : 1);
  k_emit<<<grid, 256, 0, st>>>(ws.rec, ws.offsets, PN, ws.n, ws.tile, ws.tiles_x, ws.T, ws.keys, ws.vals, ws.cap,
                               ws.n_pairs, ws.status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs
