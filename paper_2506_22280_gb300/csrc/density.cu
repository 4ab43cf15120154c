// Adaptive density control of the Gaussian cloud between optimisation steps (the paper's density-control
// step with its gradient threshold; the remaining rules are this library's readings, stated in
// include/digs.h): a plan kernel decides, per Gaussian, prune / keep / clone / split from the gradient
// statistic digs_step accumulates (DigsState.dens_grad), the density and the largest scale, and a prefix
// sum of the output counts (0 / 1 / 2) gives every Gaussian its first output row; an apply kernel writes
// the new cloud (clones with half the density each; split children at mu + R diag(s) z with scales
// s / 1.6 and density rho 1.6^3 / 2, z drawn by the caller); a gather kernel carries per-Gaussian rows
// (Adam moments) over, zero for new rows.
#include <algorithm>

#include "digs_internal.h"
#include "setup.cuh"

namespace digs {
namespace {

constexpr float kSplitShrink = 1.6f;

// action: -1 prune, 0 keep, 1 clone, 2 split; size: output rows of the Gaussian.
__global__ void k_dens_plan(int n, const float* __restrict__ grad_sum, const float* __restrict__ scale,
                            const float* __restrict__ rho, float thr, float s_split, float rho_min,
                            int* __restrict__ action, uint32_t* __restrict__ size) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float smax = fmaxf(fmaxf(scale[3 * i], scale[3 * i + 1]), scale[3 * i + 2]);
  int a = 0;
  if (rho[i] < rho_min) a = -1;
  else if (grad_sum[i] >= thr) a = smax > s_split ? 2 : 1;
  action[i] = a;
  size[i] = a < 0 ? 0u : (a == 0 ? 1u : 2u);
}

__global__ void k_dens_apply(int n, const float* __restrict__ mu0, const float* __restrict__ scale,
                             const float* __restrict__ quat, const float* __restrict__ rho,
                             const int* __restrict__ action, const uint32_t* __restrict__ dst,
                             const float* __restrict__ z, int cap, float* __restrict__ o_mu0,
                             float* __restrict__ o_scale, float* __restrict__ o_quat, float* __restrict__ o_rho,
                             int* __restrict__ o_src, int* __restrict__ o_new) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = action[i];
  if (a < 0) return;
  const int d = (int)dst[i];
  const int rows = a == 0 ? 1 : 2;
  const float q[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
  const float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
  float Rm[9];
  if (a == 2) {
    const float iq = 1.f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float qh[4] = {q[0] * iq, q[1] * iq, q[2] * iq, q[3] * iq};
    quat_to_R(qh, Rm);
  }
  for (int k = 0; k < rows; ++k) {
    const int j = d + k;
    if (j >= cap) return;
    float m[3] = {mu0[3 * i], mu0[3 * i + 1], mu0[3 * i + 2]}, sc[3] = {s[0], s[1], s[2]}, r = rho[i];
    if (a == 2) {
      const float* zz = z + (size_t)i * 6 + 3 * k;
      const float v0 = s[0] * zz[0], v1 = s[1] * zz[1], v2 = s[2] * zz[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        m[c] += Rm[3 * c] * v0 + Rm[3 * c + 1] * v1 + Rm[3 * c + 2] * v2;
        sc[c] = s[c] / kSplitShrink;
      }
      r = rho[i] * (kSplitShrink * kSplitShrink * kSplitShrink * 0.5f);
    } else if (a == 1) {
      r = 0.5f * rho[i];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o_mu0[3 * j + c] = m[c];
      o_scale[3 * j + c] = sc[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) o_quat[4 * j + c] = q[c];
    o_rho[j] = r;
    o_src[j] = i;
    o_new[j] = (a == 2 || (a == 1 && k == 1)) ? 1 : 0;
  }
}

__global__ void k_gather_rows(const int* __restrict__ src, const int* __restrict__ is_new, int n_out, int dim,
                              const float* __restrict__ in, float* __restrict__ out) {
  const long long total = (long long)n_out * dim;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / dim), c = (int)(t % dim);
    out[t] = is_new[j] ? 0.f : in[(size_t)src[j] * dim + c];
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace digs

using namespace digs;

extern "C" {

size_t digs_densify_workspace_size(int n) {
  if (n < 0) return 0;
  return align256((size_t)(n + 1) * 4) + align256(scan_tmp_words(n) * 4);
}

digs_status digs_densify_plan(int n, const float* grad_sum, const float* scale, const float* rho,
                              const DigsDensifyOpts* opts, int* action, int* dst, void* ws, size_t ws_bytes,
                              void* stream) {
  if (n < 0 || !opts || opts->n_projections < 1 || !dst || !ws) return DIGS_ERR_ARG;
  if (n > 0 && (!grad_sum || !scale || !rho || !action)) return DIGS_ERR_ARG;
  if (digs_densify_workspace_size(n) > ws_bytes) return DIGS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* size = (uint32_t*)ws;
  uint32_t* tmp = (uint32_t*)((char*)ws + align256((size_t)(n + 1) * 4));
  // the threshold on the sum: tau times the projections it was summed over, rounded to float once
  const float thr = (float)((double)opts->tau * (double)opts->n_projections);
  if (n > 0) {
    k_dens_plan<<<(n + 255) / 256, 256, 0, st>>>(n, grad_sum, scale, rho, thr, opts->s_split, opts->rho_min, action,
                                                  size);
    note_launches(1);
  }
  if (exclusive_scan(size, (uint32_t*)dst, n, tmp, st) != cudaSuccess) return DIGS_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

digs_status digs_densify_apply(const DigsGaussians* g, const int* action, const int* dst, const float* z, int cap,
                               float* mu0, float* scale, float* quat, float* rho, int* src, int* is_new,
                               void* stream) {
  if (!g || g->n < 0 || cap < 0) return DIGS_ERR_ARG;
  if (g->n == 0) return DIGS_OK;
  if (!g->mu0 || !g->scale || !g->quat || !g->rho || !action || !dst || !z) return DIGS_ERR_ARG;
  if (cap > 0 && (!mu0 || !scale || !quat || !rho || !src || !is_new)) return DIGS_ERR_ARG;
  k_dens_apply<<<(g->n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      g->n, g->mu0, g->scale, g->quat, g->rho, action, (const uint32_t*)dst, z, cap, mu0, scale, quat, rho, src,
      is_new);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

digs_status digs_gather_rows(const int* src, const int* is_new, int n_out, int dim, const float* in, float* out,
                             void* stream) {
  if (n_out < 0 || dim < 1) return DIGS_ERR_ARG;
  if (n_out == 0) return DIGS_OK;
  if (!src || !is_new || !in || !out) return DIGS_ERR_ARG;
  const long long total = (long long)n_out * dim;
  const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 16);
  k_gather_rows<<<grid, 256, 0, (cudaStream_t)stream>>>(src, is_new, n_out, dim, in, out);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? DIGS_OK : DIGS_ERR_CUDA;
}

}  // extern "C"
