// Temporal B-spline of the low-rank weights (Sec. 4.2: the time axis is a cubic B-spline with control
// points every few time points, like the spatial grid of Sec. 3.3).  Projection p sits at
// tau = p / t_step + 1 in control-point units, so with f = floor(tau) - 1 and u = tau - floor(tau)
//   w_r(p) = sum_{l=0..3} B_l(u) c[f + l][r],
// B_l the uniform cubic basis of Eq. 10; control points outside [0, n_ctrl) read as zero.
#include "digs_internal.h"

namespace digs {

__device__ __forceinline__ void tbasis(float u, float B[4]) {
  const float v = 1.f - u, u2 = u * u, u3 = u2 * u;
  B[0] = v * v * v * (1.f / 6.f);
  B[1] = (3.f * u3 - 6.f * u2 + 4.f) * (1.f / 6.f);
  B[2] = (-3.f * u3 + 3.f * u2 + 3.f * u + 1.f) * (1.f / 6.f);
  B[3] = u3 * (1.f / 6.f);
}

__device__ __forceinline__ int tcell(int p, float t_step, float& u) {
  const float tau = (float)p / t_step + 1.f;
  const float fl = floorf(tau);
  u = tau - fl;
  return (int)fl - 1;
}

// w[rows[b]][r] for the B projections of a step, one thread per (b, r).
__global__ void k_temporal_eval(const float* __restrict__ ctrl, int n_ctrl, int R, float t_step,
                                const __grid_constant__ RowsParam rows, int B, float* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * R) return;
  const int b = i / R, r = i % R, p = rows.v[b];
  float u, Bw[4];
  const int f = tcell(p, t_step, u);
  tbasis(u, Bw);
  float s = 0.f;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int j = f + l;
    if (j >= 0 && j < n_ctrl) s = fmaf(Bw[l], ctrl[(size_t)j * R + r], s);
  }
  w[(size_t)p * R + r] = s;
}

// dL/dc[j][r] = sum over the step's projections b of B_{j - f_b}(u_b) dL/dw[rows[b]][r]; one thread per
// (j, r), the projections in order (no atomics).  Rows repeated in `rows` carry their gradient once.
__global__ void k_temporal_bwd(const float* __restrict__ g_w, int n_ctrl, int R, float t_step,
                               const __grid_constant__ RowsParam rows, int B, float* __restrict__ g_ctrl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ctrl * R) return;
  const int j = i / R, r = i % R;
  float s = 0.f;
  for (int b = 0; b < B; ++b) {
    const int p = rows.v[b];
    bool first = true;
    for (int q = 0; q < b; ++q) first = first && rows.v[q] != p;
    if (!first) continue;
    float u, Bw[4];
    const int f = tcell(p, t_step, u);
    const int l = j - f;
    if (l < 0 || l > 3) continue;
    tbasis(u, Bw);
    s = fmaf(l == 0 ? Bw[0] : l == 1 ? Bw[1] : l == 2 ? Bw[2] : Bw[3], g_w[(size_t)p * R + r], s);
  }
  g_ctrl[i] = s;
}

cudaError_t launch_temporal_eval(const float* ctrl, int n_ctrl, int R, float t_step, const RowsParam& rows, int B,
                                 float* w, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_temporal_eval<<<(B * R + 127) / 128, 128, 0, st>>>(ctrl, n_ctrl, R, t_step, rows, B, w);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_temporal_bwd(const float* g_w, int n_ctrl, int R, float t_step, const RowsParam& rows, int B,
                                float* g_ctrl, cudaStream_t st) {
  if (n_ctrl <= 0) return cudaSuccess;
  k_temporal_bwd<<<(n_ctrl * R + 127) / 128, 128, 0, st>>>(g_w, n_ctrl, R, t_step, rows, B, g_ctrl);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs
