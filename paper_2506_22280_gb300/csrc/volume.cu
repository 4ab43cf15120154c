// Evaluation volumes at one time point: the attenuation volume of the deformed cloud (Eq. 3 with the warp
// of Eq. 7-8), for image metrics, and the displacement field D(x, t) - x = sum_r w_r u_r(x) (Eq. 9-10),
// for motion metrics.
#include "digs_internal.h"
#include "ffd.cuh"
#include "setup.cuh"

namespace digs {
namespace {

struct GridC {
  int nx, ny, nz;
  float origin[3], spacing[3];
};

// One warp per Gaussian: deformed mean and precision factor A (Sigma'^-1 = A^T A), the axis-aligned box
// of its cutoff ellipsoid (half extents cutoff sqrt(Sigma'_ii)), then the lanes sweep the box's voxels
// and add rho exp(-E / 2) where E <= cutoff^2 (float atomics: several Gaussians share voxels).
template <int R>
__global__ void __launch_bounds__(256) k_voxelize(GaussPtrs g, LatticeC L, const float* __restrict__ phi,
                                                  const float* __restrict__ w, GridC G, float c2,
                                                  float* __restrict__ vol) {
  const int lane = threadIdx.x & 31;
  const int n = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (n >= g.n) return;
  float mu0[3], s[3], q[4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mu0[c] = g.mu0[3 * n + c];
    s[c] = g.scale[3 * n + c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] = g.quat[4 * n + c];
  const float qn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] *= qn;
  float Rm[9];
  quat_to_R(q, Rm);
  float U[R][3], dU[R][9];
  ffd_eval_point<R>(phi, L, mu0, U, dU);
  float mu[3] = {mu0[0], mu0[1], mu0[2]}, K[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float wr = w[r];
#pragma unroll
    for (int c = 0; c < 3; ++c) mu[c] = fmaf(wr, U[r][c], mu[c]);
#pragma unroll
    for (int c = 0; c < 9; ++c) K[c] = fmaf(wr, dU[r][c], K[c]);
  }
  float Ki[9], A[9];
  if (!(inv3(K, Ki) > DIGS_FOLD_EPS)) return;  // folded: dropped, as in the projector
  const float inv_s[3] = {1.f / s[0], 1.f / s[1], 1.f / s[2]};
  make_A(inv_s, Rm, Ki, A);
  // Sigma' = M M^T with M = K R S
  float half[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float m = (K[3 * i] * Rm[k] + K[3 * i + 1] * Rm[3 + k] + K[3 * i + 2] * Rm[6 + k]) * s[k];
      v = fmaf(m, m, v);
    }
    half[i] = sqrtf(c2 * v);
  }
  // P = A^T A (symmetric)
  float P[6];
  {
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int a = ij[e][0], b = ij[e][1];
      P[e] = A[a] * A[b] + A[3 + a] * A[3 + b] + A[6 + a] * A[6 + b];
    }
  }
  const int dims[3] = {G.nx, G.ny, G.nz};
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = max(0, (int)ceilf((mu[a] - half[a] - G.origin[a]) / G.spacing[a]));
    hi[a] = min(dims[a] - 1, (int)floorf((mu[a] + half[a] - G.origin[a]) / G.spacing[a]));
    if (lo[a] > hi[a]) return;
  }
  const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
  const long long count = (long long)ex * ey * ez;
  const float rho = g.rho[n];
  for (long long v = lane; v < count; v += 32) {
    const int i = lo[0] + (int)(v % ex), j = lo[1] + (int)((v / ex) % ey), k = lo[2] + (int)(v / ((long long)ex * ey));
    const float dx = G.origin[0] + i * G.spacing[0] - mu[0];
    const float dy = G.origin[1] + j * G.spacing[1] - mu[1];
    const float dz = G.origin[2] + k * G.spacing[2] - mu[2];
    const float E = P[0] * dx * dx + P[1] * dy * dy + P[2] * dz * dz +
                    2.f * (P[3] * dx * dy + P[4] * dx * dz + P[5] * dy * dz);
    if (E <= c2) atomicAdd(vol + ((size_t)k * G.ny + j) * G.nx + i, rho * __expf(-0.5f * E));
  }
}

template <int R>
__global__ void __launch_bounds__(128) k_dvf(LatticeC L, const float* __restrict__ phi, const float* __restrict__ w,
                                             GridC G, float* __restrict__ out) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nv = (long long)G.nx * G.ny * G.nz;
  if (v >= nv) return;
  const int i = (int)(v % G.nx), j = (int)((v / G.nx) % G.ny), k = (int)(v / ((long long)G.nx * G.ny));
  const float x[3] = {G.origin[0] + i * G.spacing[0], G.origin[1] + j * G.spacing[1], G.origin[2] + k * G.spacing[2]};
  float U[R][3], dU[R][9];
  ffd_eval_point<R>(phi, L, x, U, dU);
  float d[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float wr = w[r];
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = fmaf(wr, U[r][c], d[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) out[3 * v + c] = d[c];
}

bool make_grid(const DigsGrid* g, GridC& G) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  G.nx = g->nx; G.ny = g->ny; G.nz = g->nz;
  for (int a = 0; a < 3; ++a) {
    if (!(g->spacing[a] > 0.f) || !isfinite(g->spacing[a]) || !isfinite(g->origin[a])) return false;
    G.origin[a] = g->origin[a];
    G.spacing[a] = g->spacing[a];
  }
  return true;
}

bool make_lat(const DigsLattice* lat, LatticeC& L) {
  if (!lat || lat->R < 1 || lat->R > DIGS_MAX_R || lat->nx < 1 || lat->ny < 1 || lat->nz < 1) return false;
  for (int a = 0; a < 3; ++a) {
    if (!(lat->spacing[a] > 0.f) || !isfinite(lat->spacing[a]) || !isfinite(lat->origin[a])) return false;
    L.origin[a] = lat->origin[a];
    L.inv_h[a] = 1.f / lat->spacing[a];
  }
  L.nx = lat->nx; L.ny = lat->ny; L.nz = lat->nz; L.R = lat->R;
  return true;
}

}  // namespace
}  // namespace digs

using namespace digs;

extern "C" {

digs_status digs_voxelize(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                          const DigsGrid* grid, const DigsOpts* opts, float* vol, void* stream) {
  LatticeC L;
  GridC G;
  if (!g || !phi || !w || !vol || g->n < 0 || !make_lat(lat, L) || !make_grid(grid, G)) return DIGS_ERR_ARG;
  if (g->n > 0 && (!g->mu0 || !g->scale || !g->quat || !g->rho)) return DIGS_ERR_ARG;
  const float cut = opts ? opts->cutoff : 3.5f;
  if (!(cut >= 0.f) || !isfinite(cut)) return DIGS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(vol, 0, (size_t)G.nx * G.ny * G.nz * sizeof(float), st) != cudaSuccess) return DIGS_ERR_CUDA;
  if (g->n == 0) return DIGS_OK;
  GaussPtrs gp{g->mu0, g->scale, g->quat, g->rho, g->n};
  const unsigned blocks = (unsigned)(((long long)g->n * 32 + 255) / 256);
  switch (L.R) {
    case 1: k_voxelize<1><<<blocks, 256, 0, st>>>(gp, L, phi, w, G, cut * cut, vol); break;
    case 2: k_voxelize<2><<<blocks, 256, 0, st>>>(gp, L, phi, w, G, cut * cut, vol); break;
    case 3: k_voxelize<3><<<blocks, 256, 0, st>>>(gp, L, phi, w, G, cut * cut, vol); break;
    case 4: k_voxelize<4><<<blocks, 256, 0, st>>>(gp, L, phi, w, G, cut * cut, vol); break;
  }
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

digs_status digs_dvf(const DigsLattice* lat, const float* phi, const float* w, const DigsGrid* grid, float* dvf,
                     void* stream) {
  LatticeC L;
  GridC G;
  if (!phi || !w || !dvf || !make_lat(lat, L) || !make_grid(grid, G)) return DIGS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nv = (long long)G.nx * G.ny * G.nz;
  const unsigned blocks = (unsigned)((nv + 127) / 128);
  switch (L.R) {
    case 1: k_dvf<1><<<blocks, 128, 0, st>>>(L, phi, w, G, dvf); break;
    case 2: k_dvf<2><<<blocks, 128, 0, st>>>(L, phi, w, G, dvf); break;
    case 3: k_dvf<3><<<blocks, 128, 0, st>>>(L, phi, w, G, dvf); break;
    case 4: k_dvf<4><<<blocks, 128, 0, st>>>(L, phi, w, G, dvf); break;
  }
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

}  // extern "C"
