// Per-Gaussian backward chain: record gradients (summed over the Gaussian's tile slots) -> deformed mean
// and precision factor A -> K, S, R -> reference Gaussian; then through the DI warp (Eq. 7-8) and the
// FFD (Eq. 9-11) to the control points phi and the temporal weights w.
#include "digs_internal.h"
#include "ffd.cuh"
#include "setup.cuh"

namespace digs {

constexpr int kChainThreads = 128;

template <int R>
__global__ void __launch_bounds__(kChainThreads) k_chain_bwd(
    GaussPtrs g, LatticeC L, const float* __restrict__ phi, const float* __restrict__ w,
    const __grid_constant__ ViewsParam views, int P, float c2, const uint32_t* __restrict__ offsets,
    long long cap, const float4* __restrict__ partials, float* __restrict__ g_mu0, float* __restrict__ g_scale,
    float* __restrict__ g_quat, float* __restrict__ g_rho, float* __restrict__ g_phi, float* __restrict__ gw_part) {
  __shared__ float red[kChainThreads / 32][R];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = n < g.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float mu0[3] = {0.f, 0.f, 0.f}, s[3] = {1.f, 1.f, 1.f}, inv_s[3] = {1.f, 1.f, 1.f}, qh[4] = {1.f, 0.f, 0.f, 0.f};
  float qnorm = 1.f, Rm[9], rho = 0.f;
  if (valid) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mu0[c] = g.mu0[3 * n + c];
      s[c] = g.scale[3 * n + c];
      inv_s[c] = 1.f / s[c];
    }
    float q[4] = {g.quat[4 * n], g.quat[4 * n + 1], g.quat[4 * n + 2], g.quat[4 * n + 3]};
    qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
#pragma unroll
    for (int c = 0; c < 4; ++c) qh[c] = q[c] / qnorm;
    rho = g.rho[n];
  }
  quat_to_R(qh, Rm);
  float U[R][3], dU[R][9];
  if (valid) {
    ffd_eval_point<R>(phi, L, mu0, U, dU);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int c = 0; c < 3; ++c) U[r][c] = 0.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) dU[r][c] = 0.f;
    }
  }
  float GU[R][3], GdU[R][9];
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) GU[r][c] = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) GdU[r][c] = 0.f;
  }
  float gmu0[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gR[9], grho = 0.f;
#pragma unroll
  for (int c = 0; c < 9; ++c) gR[c] = 0.f;

  for (int b = 0; b < P; ++b) {
    const ViewC& v = views.v[b];
    float gw[R];
#pragma unroll
    for (int r = 0; r < R; ++r) gw[r] = 0.f;
    size_t idx = (size_t)b * g.n + n;
    uint32_t off = valid ? offsets[idx] : 0u, end = valid ? offsets[idx + 1] : 0u;
    if ((long long)end > cap) end = (uint32_t)cap;  // pairs past the capacity were never binned
    if (off > end) off = end;
    if (off != end) {
      const float* wb = w + (size_t)v.w_row * R;
      float wr[R], mu[3], K[9];
#pragma unroll
      for (int c = 0; c < 3; ++c) mu[c] = mu0[c];
#pragma unroll
      for (int c = 0; c < 9; ++c) K[c] = (c % 4 == 0) ? 1.f : 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        wr[r] = __ldg(wb + r);
#pragma unroll
        for (int c = 0; c < 3; ++c) mu[c] = fmaf(wr[r], U[r][c], mu[c]);
#pragma unroll
        for (int c = 0; c < 9; ++c) K[c] = fmaf(wr[r], dU[r][c], K[c]);
      }
      float Ki[9], A[9];
      inv3(K, Ki);
      make_A(inv_s, Rm, Ki, A);
      SetupState st;
      setup_core(v, mu, A, rho, st);
      // sum the backward partials of this (projection, Gaussian) over its tiles, in slot order
      float S[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) S[q] = 0.f;
      for (uint32_t k = off; k < end; ++k) {
        const float4* p = partials + (size_t)k * DIGS_PARTIAL_F4;
        float4 a = p[0], c = p[1], d = p[2];
        S[0] += a.x; S[1] += a.y; S[2] += a.z; S[3] += a.w;
        S[4] += c.x; S[5] += c.y; S[6] += c.z; S[7] += c.w;
        S[8] += d.x; S[9] += d.y;
      }
      // record-parameter gradients (see the raster's pair formulas)
      float g_amp = S[0];
      float g_n00 = S[1], g_n01 = 2.f * S[2], g_n11 = S[3];
      float g_w0 = -S[7], g_w1 = -S[8];
      float g_kappa = S[9];
      float g_xc = -(2.f * (st.n00 * S[4] + st.n01 * S[5]) - st.w0 * S[6]);
      float g_yc = -(2.f * (st.n01 * S[4] + st.n11 * S[5]) - st.w1 * S[6]);
      float gmu[3], gA[9], grho_b;
      setup_adjoint(v, st, rho, g_xc, g_yc, g_n00, g_n01, g_n11, g_w0, g_w1, g_kappa, g_amp, gmu, gA, grho_b);
      grho += grho_b;
      // A = S^-1 R^T K^-1
#pragma unroll
      for (int i = 0; i < 3; ++i)
        gs[i] -= inv_s[i] * (gA[3 * i] * A[3 * i] + gA[3 * i + 1] * A[3 * i + 1] + gA[3 * i + 2] * A[3 * i + 2]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
          gR[3 * a + bb] += inv_s[bb] * (gA[3 * bb] * Ki[3 * a] + gA[3 * bb + 1] * Ki[3 * a + 1] + gA[3 * bb + 2] * Ki[3 * a + 2]);
      // g_K = -A^T gA K^-T
      float Tm[9], gK[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) Tm[3 * a + j] = A[a] * gA[j] + A[3 + a] * gA[3 + j] + A[6 + a] * gA[6 + j];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
          gK[3 * a + bb] = -(Tm[3 * a] * Ki[3 * bb] + Tm[3 * a + 1] * Ki[3 * bb + 1] + Tm[3 * a + 2] * Ki[3 * bb + 2]);
      // mu' = mu0 + sum_r w_r U_r, K = I + sum_r w_r dU_r
#pragma unroll
      for (int c = 0; c < 3; ++c) gmu0[c] += gmu[c];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          GU[r][c] = fmaf(wr[r], gmu[c], GU[r][c]);
          acc = fmaf(gmu[c], U[r][c], acc);
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          GdU[r][c] = fmaf(wr[r], gK[c], GdU[r][c]);
          acc = fmaf(gK[c], dU[r][c], acc);
        }
        gw[r] = acc;
      }
    }
    // deterministic block reduction of dL/dw[b][r]
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float t = warp_sum(gw[r]);
      if (lane == 0) red[warp][r] = t;
    }
    __syncthreads();
    if (threadIdx.x < R) {
      float t = 0.f;
#pragma unroll
      for (int ww = 0; ww < kChainThreads / 32; ++ww) t += red[ww][threadIdx.x];
      gw_part[((size_t)blockIdx.x * P + b) * R + threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (!valid) return;
  ffd_bwd_point<R>(phi, g_phi, L, mu0, GU, GdU, gmu0);
  float gq[4];
  quat_bwd(qh, qnorm, gR, gq);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g_mu0[3 * n + c] = gmu0[c];
    g_scale[3 * n + c] = gs[c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) g_quat[4 * n + c] = gq[c];
  g_rho[n] = grho;
}

cudaError_t launch_chain_bwd(const GaussPtrs& g, const LatticeC& L, const float* phi, const float* w,
                             const ViewsParam& views, int P, float c2, const Workspace& ws, float* g_mu0,
                             float* g_scale, float* g_quat, float* g_rho, float* g_phi, cudaStream_t st) {
  if (g.n <= 0) return cudaSuccess;
  dim3 grid((g.n + kChainThreads - 1) / kChainThreads);
#define DIGS_CH(RR)                                                                                            \
  k_chain_bwd<RR><<<grid, kChainThreads, 0, st>>>(g, L, phi, w, views, P, c2, ws.offsets, ws.cap, ws.partials, g_mu0, \
                                                  g_scale, g_quat, g_rho, g_phi, ws.gw_part)
  switch (L.R) {
    case 1: DIGS_CH(1); break;
    case 2: DIGS_CH(2); break;
    case 3: DIGS_CH(3); break;
    case 4: DIGS_CH(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef DIGS_CH
  note_launches(1);
  return cudaGetLastError();
}

// dL/dw[row][r] = sum over the Gaussian blocks of their partials, in block order.  Rows of w that no
// projection of the call uses get zero (the caller's buffer is cleared first).
__global__ void k_gw_reduce(const float* __restrict__ gw_part, int nblk, int P, int R, float* __restrict__ g_w,
                            const __grid_constant__ ViewsParam views) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * R) return;
  int b = i / R, r = i % R;
  float s = 0.f;
  for (int k = 0; k < nblk; ++k) s += gw_part[((size_t)k * P + b) * R + r];
  atomicAdd(&g_w[(size_t)views.v[b].w_row * R + r], s);  // rows repeat only if a time point repeats
}

cudaError_t launch_gw_reduce(const Workspace& ws, const ViewsParam& views, int P, int R, float* g_w, int w_rows,
                             cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g_w, 0, sizeof(float) * (size_t)w_rows * R, st);
  if (e != cudaSuccess || P * R == 0) return e;
  int nblk = ws.n > 0 ? (ws.n + kChainThreads - 1) / kChainThreads : 0;
  if (nblk == 0) return cudaSuccess;
  k_gw_reduce<<<(P * R + 127) / 128, 128, 0, st>>>(ws.gw_part, nblk, P, R, g_w, views);
  note_launches(1);
  return cudaGetLastError();
}

int chain_blocks(int n) { return (n + kChainThreads - 1) / kChainThreads; }

}  // namespace digs
