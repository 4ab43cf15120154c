// Per-Gaussian backward chain: record gradients (the raster backward's ten sums per pair) -> deformed mean
// and precision factor A -> K, S, R -> reference Gaussian; then through the DI warp (Eq. 7-8) and the
// FFD (Eq. 9-11) to the control points phi and the temporal weights w.
//
// Three kernels.  (1) For 32 Gaussians per CTA, each warp takes a slot of the projections: one thread per
// (projection, Gaussian) pair takes the pair's ten pixel sums and runs the adjoint of the projection
// set-up and of A = S^-1 R^T K^-1; the pair adjoints (and their w-weighted sums, what the FFD backward
// needs) are added up per Gaussian in shared memory, and dL/dw per projection is summed over the CTA's
// Gaussians.  (2) One thread per Gaussian forms dL/du_r and dL/d(grad u_r) from those sums and scatters
// the FFD backward to the control points: when all 32 Gaussians of a warp sit in the same lattice cell
// (the usual case for spatially ordered clouds) the warp first sums its 64 x 3R values with a
// transposed shuffle reduction and issues one atomic per control-point component; otherwise each lane
// adds its own.  (3) dL/dw adds the per-CTA sums in a fixed order.
#include "digs_internal.h"
#include "ffd.cuh"
#include "setup.cuh"

namespace digs {

constexpr int kChainThreads = 128;

int chain_blocks(int n) { return (n + kChainThreads - 1) / kChainThreads; }

// Sum 48 per-lane values over the warp; lane l ends with 3 complete sums, values
// base(l) + j (j < 3) with base = 24 b4 + 12 b3 + 6 b2 + 3 b1 (b_i = bit i of l); lanes l and l^1 agree.
__device__ __forceinline__ void warp_reduce_scatter48(float v[48], int lane) {
#pragma unroll
  for (int half = 24, bit = 16; half >= 3; half >>= 1, bit >>= 1) {
    const bool hi = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      float send = hi ? v[i] : v[i + half];
      float keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 1);
}

// Scatter of the control-point gradient for a whole warp: dL/dphi_r[node]_c += beta GU_c + sum_j GdU_cj
// d_j beta for the 64 nodes around x (Eq. 10 differentiated); lanes in the same lattice cell are summed
// over the warp first.  GU / GdU: this thread's dL/du_r and
// dL/d(grad u_r), read from shared memory at stride `st`.  Lanes with valid == false contribute nothing
// but take part in the warp collectives.
template <int R>
__device__ __forceinline__ void ffd_scatter_warp(float* __restrict__ g_phi_all, long long phi_stride, int scan,
                                                 const LatticeC& L, const float x[3], bool valid, const float* GU,
                                                 const float* GdU, int st) {
  const int lane = threadIdx.x & 31;
  int f[3];
  float u[3];
  lattice_cell(L, x, f, u);
  float B[3][4], dB[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bspline4(u[a], B[a]);
    bspline4_d1(u[a], dB[a]);
#pragma unroll
    for (int l = 0; l < 4; ++l) dB[a][l] *= L.inv_h[a];
  }
  const unsigned long long key =
      valid ? ((unsigned long long)((unsigned)(f[0] + 1024) | ((unsigned)(f[1] + 1024) << 11) |
                                    ((unsigned)(f[2] + 512) << 22)) |
               ((unsigned long long)scan << 32))
            : ~0ull - (unsigned long long)lane;
  float* g_phi = g_phi_all + scan * phi_stride;
  // Lanes sharing a scan and a lattice cell share the 64 nodes: group them (up to 4 groups per warp) and
  // let each group sum its values over the warp before one atomic per node component.
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const unsigned leaders = __ballot_sync(0xffffffffu, (peers & ((1u << lane) - 1u)) == 0u);
  const bool grouped = __popc(leaders) <= 4;
  const size_t rank_stride = (size_t)L.nx * L.ny * L.nz * 3;
#pragma unroll 1
  for (int r = 0; r < R; ++r) {
    float gu[3], gdu[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) gu[c] = valid ? GU[(r * 3 + c) * st] : 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) gdu[c] = valid ? GdU[(r * 9 + c) * st] : 0.f;
#pragma unroll 1
    for (int n3 = 0; n3 < 4; ++n3) {
      const float bz = n3 == 0 ? B[2][0] : n3 == 1 ? B[2][1] : n3 == 2 ? B[2][2] : B[2][3];
      const float dbz = n3 == 0 ? dB[2][0] : n3 == 1 ? dB[2][1] : n3 == 2 ? dB[2][2] : dB[2][3];
      // v[(m * 4 + l) * 3 + c] = beta gu_c + sum_j gdu_cj d_j beta for node (l, m, n3); zero unless `on`
      auto slab = [&](float v[48], bool on) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            const float bx = B[0][l], by = B[1][m];
            const float beta = on ? bx * by * bz : 0.f;
            const float gb0 = on ? dB[0][l] * by * bz : 0.f, gb1 = on ? bx * dB[1][m] * bz : 0.f;
            const float gb2 = on ? bx * by * dbz : 0.f;
            const int q = (m * 4 + l) * 3;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              v[q + c] = beta * gu[c] + gdu[3 * c] * gb0 + gdu[3 * c + 1] * gb1 + gdu[3 * c + 2] * gb2;
          }
        }
      };
      if (grouped) {
        unsigned rem = leaders;
        while (rem) {  // warp-uniform
          const int ld = __ffs(rem) - 1;
          rem &= rem - 1u;
          const unsigned gmask = __shfl_sync(0xffffffffu, peers, ld);
          const int gi = __shfl_sync(0xffffffffu, f[0], ld), gj = __shfl_sync(0xffffffffu, f[1], ld);
          const int gk = __shfl_sync(0xffffffffu, f[2], ld) + n3;
          const bool gvalid = __shfl_sync(0xffffffffu, valid ? 1 : 0, ld) != 0;
          float* gphi = g_phi_all + __shfl_sync(0xffffffffu, scan, ld) * phi_stride;
          float v[48];
          slab(v, ((gmask >> lane) & 1u) != 0u);
          warp_reduce_scatter48(v, lane);
          if ((lane & 1) == 0 && gvalid && gk >= 0 && gk < L.nz) {
            const int base = ((lane >> 4) & 1) * 24 + ((lane >> 3) & 1) * 12 + ((lane >> 2) & 1) * 6 + ((lane >> 1) & 1) * 3;
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
              const int idx = base + jj, node = idx / 3, c = idx % 3;
              const int i = gi + (node & 3), j = gj + (node >> 2);
              if (i >= 0 && i < L.nx && j >= 0 && j < L.ny)
                atomicAdd(gphi + r * rank_stride + (((size_t)gk * L.ny + j) * L.nx + i) * 3 + c, v[jj]);
            }
          }
        }
      } else {
        const int k = f[2] + n3;
        if (valid && k >= 0 && k < L.nz) {
          float v[48];
          slab(v, true);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int j = f[1] + m;
            if (j < 0 || j >= L.ny) continue;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              const int i = f[0] + l;
              if (i < 0 || i >= L.nx) continue;
              float* gp = g_phi + r * rank_stride + (((size_t)k * L.ny + j) * L.nx + i) * 3;
              const int q = (m * 4 + l) * 3;
              atomicAdd(gp, v[q]);
              atomicAdd(gp + 1, v[q + 1]);
              atomicAdd(gp + 2, v[q + 2]);
            }
          }
        }
      }
    }
  }
}

// Adjoint of one (projection b, Gaussian n) pair from its ten pixel sums S: dL/dmu' (gmu), dL/dK (gK),
// dL/ds (gs), dL/dtheta (gth: the gradient for a rotation R -> R (I + [theta]x) of the Gaussian's own
// axes), dL/drho (grho) and dL/dw_r (gw).  mu0, sc = s, inv_s = 1 / s, Rm, rho: the Gaussian.
//
// The record depends on A = S^-1 R^T K^-1 only through A^T A (the deformed precision), so dL/dA = 2 A G
// with G symmetric and C = A dL/dA^T is symmetric.  The rotation moves A by -S^-1 [theta]x S A, hence
// dL/dtheta_i = -C_jk (s_j / s_k - s_k / s_j) for (i, j, k) cyclic: the symmetric part of C times the
// scale anisotropy, both formed without cancellation, where a general dL/dR projected onto rotations
// afterwards would subtract two nearly equal FP32 numbers for nearly isotropic Gaussians.
template <int R>
__device__ __forceinline__ void pair_adjoint(const ViewC& v, const float* __restrict__ ffd, int N, int n,
                                             const float* wr, const float mu0[3], const float sc[3],
                                             const float inv_s[3], const float Rm[9], float rho, const float S[10],
                                             float gmu[3], float gK[9], float gs[3], float gth[3], float& grho,
                                             float gw[R]) {
  float mu[3], K[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) mu[c] = mu0[c];
#pragma unroll
  for (int c = 0; c < 9; ++c) K[c] = (c % 4 == 0) ? 1.f : 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) mu[c] = fmaf(wr[r], __ldg(ffd + (size_t)(r * 3 + c) * N + n), mu[c]);
#pragma unroll
    for (int c = 0; c < 9; ++c) K[c] = fmaf(wr[r], __ldg(ffd + (size_t)(3 * R + r * 9 + c) * N + n), K[c]);
  }
  float Ki[9], A[9];
  inv3(K, Ki);
  make_A(inv_s, Rm, Ki, A);
  float gA[9];
  // record-parameter gradients (see the raster's pair formulas)
  if (v.ewa) {  // the 2D-Gaussian model: w = kappa = 0
    EwaState es;
    ewa_core(v, mu, A, rho, es);
    const float id = 1.f / es.det2, n00 = es.s11 * id, n01 = -es.s01 * id, n11 = es.s00 * id;
    const float g_xc = -2.f * (n00 * S[4] + n01 * S[5]), g_yc = -2.f * (n01 * S[4] + n11 * S[5]);
    ewa_adjoint(v, es, rho, g_xc, g_yc, S[1], 2.f * S[2], S[3], S[0], gmu, gA, grho);
  } else {
    SetupState st;
    setup_core(v, mu, A, rho, st);
    const float g_xc = -(2.f * (st.n00 * S[4] + st.n01 * S[5]) - st.w0 * S[6]);
    const float g_yc = -(2.f * (st.n01 * S[4] + st.n11 * S[5]) - st.w1 * S[6]);
    setup_adjoint(v, st, rho, g_xc, g_yc, S[1], 2.f * S[2], S[3], -S[7], -S[8], S[9], S[0], gmu, gA, grho);
  }
  // A = S^-1 R^T K^-1: dL/ds, dL/dR, dL/dK = -A^T gA K^-T
#pragma unroll
  for (int ii = 0; ii < 3; ++ii)
    gs[ii] = -inv_s[ii] * (gA[3 * ii] * A[3 * ii] + gA[3 * ii + 1] * A[3 * ii + 1] + gA[3 * ii + 2] * A[3 * ii + 2]);
  {
    auto csym = [&](int i, int j) {  // (C_ij + C_ji) / 2, C_ij = A_i . (dL/dA)_j (rows)
      return 0.5f * (A[3 * i] * gA[3 * j] + A[3 * i + 1] * gA[3 * j + 1] + A[3 * i + 2] * gA[3 * j + 2] +
                     A[3 * j] * gA[3 * i] + A[3 * j + 1] * gA[3 * i + 1] + A[3 * j + 2] * gA[3 * i + 2]);
    };
    auto aniso = [&](int j, int k) { return (sc[j] - sc[k]) * (sc[j] + sc[k]) * inv_s[j] * inv_s[k]; };
    gth[0] = -csym(1, 2) * aniso(1, 2);
    gth[1] = -csym(2, 0) * aniso(2, 0);
    gth[2] = -csym(0, 1) * aniso(0, 1);
  }
  {
    float Tm[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) Tm[3 * a + j] = A[a] * gA[j] + A[3 + a] * gA[3 + j] + A[6 + a] * gA[6 + j];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
        gK[3 * a + bb] = -(Tm[3 * a] * Ki[3 * bb] + Tm[3 * a + 1] * Ki[3 * bb + 1] + Tm[3 * a + 2] * Ki[3 * bb + 2]);
  }
  // dL/dw_r = dL/dmu' . u_r + dL/dK : grad u_r
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc = fmaf(gmu[c], __ldg(ffd + (size_t)(r * 3 + c) * N + n), acc);
#pragma unroll
    for (int c = 0; c < 9; ++c) acc = fmaf(gK[c], __ldg(ffd + (size_t)(3 * R + r * 9 + c) * N + n), acc);
    gw[r] = acc;
  }
}

// (1) Per Gaussian, the pair adjoints summed over its projections.  A CTA takes 32 Gaussians (its lanes)
// and kSlots projection slots (its warps): warp k handles projections k, k + kSlots, ..., each thread
// adding its pair's adjoint into its own shared-memory column; the slots are then summed in order.
// gsum [11 + 12 R][N]: dL/dmu' (3), dL/ds (3), dL/dtheta (3), dL/drho (1), sum_b w_br dL/dmu'_b (3R),
// sum_b w_br dL/dK_b (9R) and sum_b |dL/dmu'_b| (the density-control statistic).  gw_part [CTA][P][R]: dL/dw_r of each projection summed over the CTA's
// Gaussians (a warp sum; each (CTA, projection) is written by one warp).
constexpr int kSlots = 8;
template <int R>
__host__ __device__ constexpr int gauss_sum_count() { return 11 + 12 * R; }
template <int R>
constexpr size_t pair_sum_smem() { return (size_t)gauss_sum_count<R>() * kSlots * 32 * sizeof(float); }
int pair_sum_blocks(int n) { return (n + 31) / 32; }

template <int R>
__global__ void __launch_bounds__(kSlots * 32, 2) k_pair_sum(GaussPtrs g, const __grid_constant__ ScanTable sc,
                                                             const float* __restrict__ ffd, const float* __restrict__ w,
                                                             const __grid_constant__ ViewsParam views, int P,
                                                             const uint32_t* __restrict__ counts,
                                                             const float4* __restrict__ sums, float* __restrict__ gsum,
                                                             float* __restrict__ gw_part) {
  constexpr int Q = gauss_sum_count<R>(), QS = kSlots * 32;
  extern __shared__ float acc[];  // [Q][kSlots][32]
  const int lane = threadIdx.x & 31, slot = threadIdx.x >> 5;
  const int N = g.n, NM = sc.nmax;
  const int n = blockIdx.x * 32 + lane;
  const bool valid = n < N;
  const int scan = valid ? scan_of(sc, n) : 0, nl = n - sc.off[scan];
  float* my = acc + slot * 32 + lane;
  if (slot >= P) {  // a slot with no projection keeps a zero column
#pragma unroll
    for (int q = 0; q < Q; ++q) my[q * QS] = 0.f;
  }
  float mu0[3] = {0.f, 0.f, 0.f}, scl[3] = {1.f, 1.f, 1.f}, inv_s[3] = {1.f, 1.f, 1.f}, Rm[9], rho = 0.f;
  if (valid) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      mu0[c] = g.mu0[3 * n + c];
      scl[c] = g.scale[3 * n + c];
      inv_s[c] = 1.f / scl[c];
    }
    const float q0 = g.quat[4 * n], q1 = g.quat[4 * n + 1], q2 = g.quat[4 * n + 2], q3 = g.quat[4 * n + 3];
    const float iq = 1.f / sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float qh[4] = {q0 * iq, q1 * iq, q2 * iq, q3 * iq};
    quat_to_R(qh, Rm);
    rho = g.rho[n];
  }
  for (int b0 = 0; b0 < P; b0 += kSlots) {
    const int b = b0 + slot;  // the same for the whole warp
    if (b >= P) break;
    const ViewC& v = views.v[b];
    const float* wb = w + (size_t)v.w_row * R;
    float gw[R];
#pragma unroll
    for (int r = 0; r < R; ++r) gw[r] = 0.f;
    const size_t i = (size_t)b * NM + nl;
    const bool first = b0 == 0;  // the slot's first projection writes its column, later ones add to it
    auto put = [&](int q, float x) {
      if (first) my[q * QS] = x;
      else my[q * QS] += x;
    };
    if (valid && v.scan == scan && counts[i] != 0u) {  // else the pair was culled by the projection set-up
      float S[10];
      {
        const float4* p = sums + i * DIGS_PARTIAL_F4;
        const float4 a = p[0], c = p[1], d = p[2];
        S[0] = a.x; S[1] = a.y; S[2] = a.z; S[3] = a.w;
        S[4] = c.x; S[5] = c.y; S[6] = c.z; S[7] = c.w;
        S[8] = d.x; S[9] = d.y;
      }
      float wr[R], gmu[3], gK[9], gs[3], gth[3], grho;
#pragma unroll
      for (int r = 0; r < R; ++r) wr[r] = __ldg(wb + r);
      pair_adjoint<R>(v, ffd, N, n, wr, mu0, scl, inv_s, Rm, rho, S, gmu, gK, gs, gth, grho, gw);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        put(c, gmu[c]);
        put(3 + c, gs[c]);
        put(6 + c, gth[c]);
      }
      put(9, grho);
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) put(10 + 3 * r + c, wr[r] * gmu[c]);
#pragma unroll
        for (int c = 0; c < 9; ++c) put(10 + 3 * R + 9 * r + c, wr[r] * gK[c]);
      }
      put(10 + 12 * R, sqrtf(gmu[0] * gmu[0] + gmu[1] * gmu[1] + gmu[2] * gmu[2]));
    } else if (first) {
#pragma unroll
      for (int q = 0; q < Q; ++q) my[q * QS] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float t = warp_sum(gw[r]);
      if (lane == 0) gw_part[((size_t)blockIdx.x * P + b) * R + r] = t;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Q * 32; o += QS) {
    const int q = o >> 5, l = o & 31, nn = blockIdx.x * 32 + l;
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) t += acc[q * QS + k * 32 + l];
    if (nn < N) gsum[(size_t)q * N + nn] = t;
  }
}

// Second derivatives of u_r at each mean ([18 R][n], see ffd_hessian_rank), for the mean's gradient:
// one thread per (Gaussian, rank), the rank from blockIdx.y.
__global__ void __launch_bounds__(128) k_ffd_hessian(GaussPtrs g, const __grid_constant__ ScanTable sc, LatticeC L,
                                                    const float* __restrict__ phi, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.n) return;
  const int r = blockIdx.y;
  const float x[3] = {g.mu0[3 * n], g.mu0[3 * n + 1], g.mu0[3 * n + 2]};
  float H[18];
  const size_t rank_stride = (size_t)L.nx * L.ny * L.nz * 3;
  ffd_hessian_rank(phi + scan_of(sc, n) * sc.phi_stride + r * rank_stride, L, x, H);
#pragma unroll
  for (int c = 0; c < 18; ++c) out[(size_t)(r * 18 + c) * g.n + n] = H[c];
}

// (2) Per Gaussian: from the summed pair adjoints, the FFD backward and the reference-parameter gradients.
template <int R>
__global__ void __launch_bounds__(32 * R, 4) k_gauss_bwd(
    GaussPtrs g, const __grid_constant__ ScanTable sc, LatticeC L, const float* __restrict__ ffd,
    const float* __restrict__ ffd2,
    const float* __restrict__ gsum, float* __restrict__ dens_grad, float* __restrict__ g_mu0,
    float* __restrict__ g_scale, float* __restrict__ g_quat, float* __restrict__ g_rho, float* __restrict__ g_phi) {
  // warp r takes rank r of the CTA's 32 Gaussians: dL/du_r (3) then dL/d(grad u_r) (9), lane-fastest
  __shared__ float Gs[R][12 * 32];
  __shared__ float gpart[R][3][32];  // each rank's share of dL/dmu0
  const int N = g.n;
  const int lane = threadIdx.x & 31, r = (int)(threadIdx.x >> 5);
  const int n = blockIdx.x * 32 + lane;
  const bool valid = n < N;
  const int scan = valid ? scan_of(sc, n) : 0;
  float GU[3] = {0.f, 0.f, 0.f}, GdU[9], gm[3] = {0.f, 0.f, 0.f}, mu0[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 9; ++c) GdU[c] = 0.f;
  if (valid) {
    const float* q = gsum + n;
#pragma unroll
    for (int c = 0; c < 3; ++c) GU[c] = q[(size_t)(10 + 3 * r + c) * N];
#pragma unroll
    for (int c = 0; c < 9; ++c) GdU[c] = q[(size_t)(10 + 3 * R + 9 * r + c) * N];
#pragma unroll
    for (int c = 0; c < 3; ++c) mu0[c] = g.mu0[3 * n + c];
    // u_r and grad u_r are evaluated at mu0: dL/dmu0 += (grad u_r)^T dL/du_r + H_r : dL/d(grad u_r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* du = ffd + (size_t)(3 * R + r * 9 + c * 3) * N + n;   // d u_rc / dx_m, m = 0..2
      const float* h = ffd2 + (size_t)(r * 18 + c * 6) * N + n;          // xx, yy, zz, xy, xz, yz
      const float hxx = h[0], hyy = h[(size_t)N], hzz = h[(size_t)2 * N];
      const float hxy = h[(size_t)3 * N], hxz = h[(size_t)4 * N], hyz = h[(size_t)5 * N];
      const float g0 = GdU[3 * c], g1 = GdU[3 * c + 1], g2 = GdU[3 * c + 2];
      gm[0] += du[0] * GU[c] + hxx * g0 + hxy * g1 + hxz * g2;
      gm[1] += du[(size_t)N] * GU[c] + hxy * g0 + hyy * g1 + hyz * g2;
      gm[2] += du[(size_t)2 * N] * GU[c] + hxz * g0 + hyz * g1 + hzz * g2;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Gs[r][c * 32 + lane] = GU[c];
    gpart[r][c][lane] = gm[c];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) Gs[r][(3 + c) * 32 + lane] = GdU[c];
  // each lane reads back only its own column of Gs[r], so no barrier is needed before the scatter
  const size_t rank_stride = (size_t)L.nx * L.ny * L.nz * 3;
  ffd_scatter_warp<1>(g_phi + r * rank_stride, sc.phi_stride, scan, L, mu0, valid, &Gs[r][lane], &Gs[r][3 * 32 + lane],
                      32);
  __syncthreads();
  if (r != 0 || !valid) return;
  const float* q = gsum + n;
  float gmu0[3], gs[3], gth[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gmu0[c] = q[(size_t)c * N];
#pragma unroll
    for (int k = 0; k < R; ++k) gmu0[c] += gpart[k][c][lane];
    gs[c] = q[(size_t)(3 + c) * N];
    gth[c] = q[(size_t)(6 + c) * N];
  }
  const float grho = q[(size_t)9 * N];
  float qh[4], gq[4];
  const float q0 = g.quat[4 * n], q1 = g.quat[4 * n + 1], q2 = g.quat[4 * n + 2], q3 = g.quat[4 * n + 3];
  const float qn = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  qh[0] = q0 / qn; qh[1] = q1 / qn; qh[2] = q2 / qn; qh[3] = q3 / qn;
  quat_bwd_rot(qh, qn, gth, gq);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g_mu0[3 * n + c] = gmu0[c];
    g_scale[3 * n + c] = gs[c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) g_quat[4 * n + c] = gq[c];
  g_rho[n] = grho;
  if (dens_grad) dens_grad[n] += gsum[(size_t)(10 + 12 * R) * N + n];  // density-control statistic
}

cudaError_t launch_chain_bwd(const GaussPtrs& g, const ScanTable& sc, const LatticeC& L, const float* phi,
                             const float* w, const ViewsParam& views, int P, const Workspace& ws, float* g_mu0,
                             float* g_scale, float* g_quat, float* g_rho, float* g_phi, float* dens_grad,
                             cudaStream_t st) {
  if (g.n <= 0) return cudaSuccess;
  dim3 gb(chain_blocks(g.n)), gp(pair_sum_blocks(g.n));
#define DIGS_CH(RR)                                                                                             \
  {                                                                                                             \
    static bool configured = false;                                                                             \
    if (!configured) {                                                                                          \
      cudaFuncSetAttribute(k_pair_sum<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_sum_smem<RR>()); \
      configured = true;                                                                                        \
    }                                                                                                           \
  }                                                                                                             \
  k_ffd_hessian<<<dim3(gb.x, RR), 128, 0, st>>>(g, sc, L, phi, ws.ffd2);                                      \
  k_pair_sum<RR><<<gp, kSlots * 32, pair_sum_smem<RR>(), st>>>(g, sc, ws.ffd, w, views, P, ws.counts, ws.grec,   \
                                                              ws.gsum, ws.gw_part);                            \
  k_gauss_bwd<RR><<<(g.n + 31) / 32, 32 * RR, 0, st>>>(g, sc, L, ws.ffd, ws.ffd2, ws.gsum, dens_grad, g_mu0,     \
                                                       g_scale,                                              \
                                               g_quat, g_rho, g_phi)
  switch (L.R) {
    case 1: DIGS_CH(1); break;
    case 2: DIGS_CH(2); break;
    case 3: DIGS_CH(3); break;
    case 4: DIGS_CH(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef DIGS_CH
  note_launches(3);
  return cudaGetLastError();
}

// (3) dL/dw[row(b)][r]: the per-CTA sums of k_pair_sum added in CTA order (strided over the block's
// threads, then a fixed-order tree), one block per (projection, rank).  Rows of w that no projection of
// the call uses get zero.
__global__ void __launch_bounds__(256) k_gw_final(const float* __restrict__ part, int n_cta, int P, int R,
                                                  float* __restrict__ g_w, const __grid_constant__ ViewsParam views) {
  __shared__ float red[8];
  const int b = blockIdx.x / R, r = blockIdx.x % R;
  float s = 0.f;
  for (int k = threadIdx.x; k < n_cta; k += blockDim.x) s += part[((size_t)k * P + b) * R + r];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k];
    atomicAdd(&g_w[(size_t)views.v[b].w_row * R + r], t);  // rows repeat only if a time point repeats
  }
}

cudaError_t launch_gw_reduce(const Workspace& ws, const ViewsParam& views, int P, int R, float* g_w, int w_rows,
                             cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g_w, 0, sizeof(float) * (size_t)w_rows * R, st);
  if (e != cudaSuccess || P * R == 0 || ws.n_total == 0) return e;
  k_gw_final<<<P * R, 256, 0, st>>>(ws.gw_part, pair_sum_blocks(ws.n_total), P, R, g_w, views);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs
