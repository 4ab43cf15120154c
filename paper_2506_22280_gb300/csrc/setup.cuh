// Per-(projection, Gaussian) set-up: rotation, deformation-informed warp (Sec. 3.2, Eq. 7-8) and the
// closed-form description of the Gaussian's ray integrals on the detector (Sec. 3.1, Eq. 4), plus the
// hand-written adjoint of all of it.
//
// Formulation.  Write the deformed precision as P' = A^T A with A = S^-1 R^T K^-1 (so P' = (K R S^2 R^T
// K^T)^-1 = Sigma'^-1 exactly, without inverting Sigma').  For a cone-beam ray from the source s through
// the detector point X_c + [e_u du, e_v dv] Delta (X_c: the detector image of the mean mu', Delta in
// pixels), with d0 = mu' - s, lambda = |X_c - s| / |d0|, alpha = A d0, Lm = |alpha|, Y = A [e_u du, e_v dv]
// / lambda, y_a = Y^T alpha / Lm and Z = (I - alpha alpha^T / Lm^2) Y, the squared Mahalanobis distance
// from the ray to mu' is E = |Z Delta|^2 / D with D = (1 - w . Delta)^2 + |Z Delta|^2 / Lm^2, w = -y_a / Lm,
// and the whole-line integral is rho sqrt(2 pi) / (lambda Lm) * |X - s| * D^-1/2 * exp(-E / 2).
// Neither expression subtracts two quantities of the source-distance scale, which keeps FP32 accurate;
// for parallel rays along u the same holds with alpha = A u, lambda = 1, D = 1 and no |X - s| factor.
#pragma once

#include "digs_common.cuh"

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_R(const float q[4], float R[9]) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// dL/dq for the gradient gth of a rotation R -> R (I + [theta]x) of the Gaussian's axes: the unit
// quaternion moves by q_hat (x) (0, theta / 2) (Hamilton product, R(q1 (x) q2) = R(q1) R(q2)), so
// dL/dq_hat = 2 q_hat (x) (0, gth), tangent to the unit sphere, and q_hat = q / |q| divides it by |q|.
__device__ __forceinline__ void quat_bwd_rot(const float qh[4], float qnorm, const float gth[3], float gq[4]) {
  const float w = qh[0], x = qh[1], y = qh[2], z = qh[3];
  const float f = 2.f / qnorm;
  gq[0] = -f * (x * gth[0] + y * gth[1] + z * gth[2]);
  gq[1] = f * (w * gth[0] + y * gth[2] - z * gth[1]);
  gq[2] = f * (w * gth[1] + z * gth[0] - x * gth[2]);
  gq[3] = f * (w * gth[2] + x * gth[1] - y * gth[0]);
}

// Inverse (row-major) by the adjugate; returns det K.
__device__ __forceinline__ float inv3(const float K[9], float Ki[9]) {
  float c0 = K[4] * K[8] - K[5] * K[7];
  float c1 = K[5] * K[6] - K[3] * K[8];
  float c2 = K[3] * K[7] - K[4] * K[6];
  float det = K[0] * c0 + K[1] * c1 + K[2] * c2;
  float id = 1.f / det;
  Ki[0] = c0 * id; Ki[1] = (K[2] * K[7] - K[1] * K[8]) * id; Ki[2] = (K[1] * K[5] - K[2] * K[4]) * id;
  Ki[3] = c1 * id; Ki[4] = (K[0] * K[8] - K[2] * K[6]) * id; Ki[5] = (K[2] * K[3] - K[0] * K[5]) * id;
  Ki[6] = c2 * id; Ki[7] = (K[1] * K[6] - K[0] * K[7]) * id; Ki[8] = (K[0] * K[4] - K[1] * K[3]) * id;
  return det;
}

// A = S^-1 R^T K^-1.
__device__ __forceinline__ void make_A(const float inv_s[3], const float R[9], const float Ki[9], float A[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      A[3 * i + j] = inv_s[i] * (R[i] * Ki[j] + R[3 + i] * Ki[3 + j] + R[6 + i] * Ki[6 + j]);
}

// Forward intermediates shared by the set-up and its adjoint.
struct SetupState {
  float mu_d[3], d0[3];
  float Ad[9];           // A expressed in the detector frame: Ad[i][c] = A[i] . frame_c
  float lam, inv_lam;
  float al[3], Lm, inv_Lm, ah[3];
  float Y0[3], Y1[3], ya0, ya1, Z0[3], Z1[3];
  float n00, n01, n11, w0, w1, kappa, amp, xc, yc;
};

__device__ __forceinline__ bool setup_core(const ViewC& v, const float mu[3], const float A[9], float rho,
                                           SetupState& s) {
#pragma unroll
  for (int c = 0; c < 3; ++c) s.mu_d[c] = v.F[3 * c] * mu[0] + v.F[3 * c + 1] * mu[1] + v.F[3 * c + 2] * mu[2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      s.Ad[3 * i + c] = A[3 * i] * v.F[3 * c] + A[3 * i + 1] * v.F[3 * c + 1] + A[3 * i + 2] * v.F[3 * c + 2];
  const float* ray;
  if (!v.parallel) {
#pragma unroll
    for (int c = 0; c < 3; ++c) s.d0[c] = s.mu_d[c] - v.src_d[c];
    if (!(s.d0[2] > 0.f)) return false;  // mean not in front of the source
    s.lam = v.sdd_n / s.d0[2];
    s.inv_lam = s.d0[2] / v.sdd_n;
    s.xc = v.cx0 + (v.su + s.lam * s.d0[0]) * v.inv_du;
    s.yc = v.cy0 + (v.sv + s.lam * s.d0[1]) * v.inv_dv;
    ray = s.d0;
  } else {
    s.lam = 1.f;
    s.inv_lam = 1.f;
    float t = (v.det_d[2] - s.mu_d[2]) / v.dir_d[2];
    s.xc = v.cx0 + (s.mu_d[0] - v.det_d[0] + t * v.dir_d[0]) * v.inv_du;
    s.yc = v.cy0 + (s.mu_d[1] - v.det_d[1] + t * v.dir_d[1]) * v.inv_dv;
    ray = v.dir_d;
  }
  float Lm2 = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.al[i] = s.Ad[3 * i] * ray[0] + s.Ad[3 * i + 1] * ray[1] + s.Ad[3 * i + 2] * ray[2];
    Lm2 += s.al[i] * s.al[i];
    s.Y0[i] = s.Ad[3 * i] * v.du * s.inv_lam;
    s.Y1[i] = s.Ad[3 * i + 1] * v.dv * s.inv_lam;
  }
  s.Lm = sqrtf(Lm2);
  s.inv_Lm = 1.f / s.Lm;
#pragma unroll
  for (int i = 0; i < 3; ++i) s.ah[i] = s.al[i] * s.inv_Lm;
  s.ya0 = s.Y0[0] * s.ah[0] + s.Y0[1] * s.ah[1] + s.Y0[2] * s.ah[2];
  s.ya1 = s.Y1[0] * s.ah[0] + s.Y1[1] * s.ah[1] + s.Y1[2] * s.ah[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.Z0[i] = s.Y0[i] - s.ah[i] * s.ya0;
    s.Z1[i] = s.Y1[i] - s.ah[i] * s.ya1;
  }
  s.n00 = s.Z0[0] * s.Z0[0] + s.Z0[1] * s.Z0[1] + s.Z0[2] * s.Z0[2];
  s.n01 = s.Z0[0] * s.Z1[0] + s.Z0[1] * s.Z1[1] + s.Z0[2] * s.Z1[2];
  s.n11 = s.Z1[0] * s.Z1[0] + s.Z1[1] * s.Z1[1] + s.Z1[2] * s.Z1[2];
  if (!v.parallel) {
    s.w0 = -s.ya0 * s.inv_Lm;
    s.w1 = -s.ya1 * s.inv_Lm;
    s.kappa = s.inv_Lm * s.inv_Lm;
  } else {
    s.w0 = s.w1 = s.kappa = 0.f;
  }
  s.amp = rho * DIGS_SQRT_2PI * s.inv_lam * s.inv_Lm;
  return isfinite(s.xc) && isfinite(s.yc) && isfinite(s.n00) && isfinite(s.n11) && isfinite(s.amp);
}

// Record plus conservative pixel box of { Delta : E(Delta) <= c2 }.  Returns false when the pair cannot
// contribute (mean behind the source, source inside the cutoff ellipsoid, box off the detector).
__device__ __forceinline__ bool setup_record(const ViewC& v, const float mu[3], const float A[9], float rho,
                                             float c2, Rec& r) {
  SetupState s;
  if (!setup_core(v, mu, A, rho, s)) return false;
  // E <= c2  <=>  Delta^T M Delta + 2 c2 w . Delta - c2 <= 0 with M = (1 - c2 kappa) N - c2 w w^T, an
  // ellipse when M is positive definite (the source lies outside the cutoff ellipsoid).
  float sc = 1.f - c2 * s.kappa;
  float m00 = sc * s.n00 - c2 * s.w0 * s.w0;
  float m01 = sc * s.n01 - c2 * s.w0 * s.w1;
  float m11 = sc * s.n11 - c2 * s.w1 * s.w1;
  float det = m00 * m11 - m01 * m01;
  if (!(m00 > 0.f) || !(det > 0.f)) return false;
  float i00 = m11 / det, i01 = -m01 / det, i11 = m00 / det;
  float mw0 = i00 * s.w0 + i01 * s.w1, mw1 = i01 * s.w0 + i11 * s.w1;
  float ox = -c2 * mw0, oy = -c2 * mw1;
  float cp = c2 + c2 * c2 * (s.w0 * mw0 + s.w1 * mw1);
  float hx = sqrtf(cp * i00) * 1.0001f + 1e-3f, hy = sqrtf(cp * i11) * 1.0001f + 1e-3f;
  float fx0 = ceilf(s.xc + ox - hx), fx1 = floorf(s.xc + ox + hx);
  float fy0 = ceilf(s.yc + oy - hy), fy1 = floorf(s.yc + oy + hy);
  fx0 = fmaxf(fx0, 0.f); fy0 = fmaxf(fy0, 0.f);
  fx1 = fminf(fx1, (float)(v.nu - 1)); fy1 = fminf(fy1, (float)(v.nv - 1));
  if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
  int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
  r.xc = s.xc; r.yc = s.yc;
  r.n00 = s.n00; r.n01x2 = 2.f * s.n01; r.n11 = s.n11;
  r.wn0 = -s.w0; r.wn1 = -s.w1; r.kappa = s.kappa; r.amp = s.amp;
  r.bx = x0 | (x1 << 16);
  r.by = y0 | (y1 << 16);
  // Bound on |D - 1| over the box for pairs inside the cutoff: |t - 1| <= tau, kappa num <= kappa c2 D.
  // When it is small, D^-1/2 = (1 + e)^-1/2 is evaluated by its binomial series through e^3 (truncation
  // below 35/128 e^4 < 5e-8 for |e| <= 0.02) instead of the SFU's rsqrt.
  float mdx = fmaxf(fabsf((float)x0 - s.xc), fabsf((float)x1 - s.xc));
  float mdy = fmaxf(fabsf((float)y0 - s.yc), fabsf((float)y1 - s.yc));
  float tau = fabsf(s.w0) * mdx + fabsf(s.w1) * mdy;
  float emax = 2.f * tau + tau * tau + 2.f * c2 * s.kappa;
  r.poly = emax <= 0.02f ? 1 : 0;
  return true;
}

// Adjoint of setup_core: from dL/d(xc, yc, n00, n01, n11, w0, w1, kappa, amp) to dL/dmu (world
// coordinates), dL/dA and dL/drho (amp = rho sqrt(2 pi) / (lambda Lm)).
__device__ __forceinline__ void setup_adjoint(const ViewC& v, const SetupState& s, float rho, float g_xc, float g_yc,
                                              float g_n00, float g_n01, float g_n11, float g_w0, float g_w1,
                                              float g_kappa, float gamp, float gmu[3], float gA[9], float& grho) {
  float gZ0[3], gZ1[3], gY0[3], gY1[3], gah[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gZ0[i] = 2.f * g_n00 * s.Z0[i] + g_n01 * s.Z1[i];
    gZ1[i] = 2.f * g_n11 * s.Z1[i] + g_n01 * s.Z0[i];
    gY0[i] = gZ0[i];
    gY1[i] = gZ1[i];
    gah[i] = -(s.ya0 * gZ0[i] + s.ya1 * gZ1[i]);
  }
  float gya0 = -(s.ah[0] * gZ0[0] + s.ah[1] * gZ0[1] + s.ah[2] * gZ0[2]);
  float gya1 = -(s.ah[0] * gZ1[0] + s.ah[1] * gZ1[1] + s.ah[2] * gZ1[2]);
  float gLm = 0.f, glam = 0.f;
  if (!v.parallel) {
    gya0 -= g_w0 * s.inv_Lm;
    gya1 -= g_w1 * s.inv_Lm;
    gLm += (g_w0 * s.ya0 + g_w1 * s.ya1) * s.inv_Lm * s.inv_Lm;
    gLm -= 2.f * g_kappa * s.inv_Lm * s.inv_Lm * s.inv_Lm;
  }
  // amp = rho sqrt(2 pi) inv_lam inv_Lm
  float ga = gamp * s.amp;  // dL/damp * amp
  grho = gamp * DIGS_SQRT_2PI * s.inv_lam * s.inv_Lm;
  gLm -= ga * s.inv_Lm;
  if (!v.parallel) glam -= ga * s.inv_lam;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gY0[i] += gya0 * s.ah[i];
    gY1[i] += gya1 * s.ah[i];
    gah[i] += gya0 * s.Y0[i] + gya1 * s.Y1[i];
  }
  float ahg = s.ah[0] * gah[0] + s.ah[1] * gah[1] + s.ah[2] * gah[2];
  float gal[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) gal[i] = (gah[i] - s.ah[i] * ahg) * s.inv_Lm + gLm * s.ah[i];
  // Y = C inv_lam, C0 = Ad[:,0] du, C1 = Ad[:,1] dv
  if (!v.parallel) {
    glam -= (gY0[0] * s.Y0[0] + gY0[1] * s.Y0[1] + gY0[2] * s.Y0[2] + gY1[0] * s.Y1[0] + gY1[1] * s.Y1[1] +
             gY1[2] * s.Y1[2]) * s.inv_lam;
  }
  float gAd[9];
  const float* ray = v.parallel ? v.dir_d : s.d0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gAd[3 * i + 0] = gal[i] * ray[0] + gY0[i] * s.inv_lam * v.du;
    gAd[3 * i + 1] = gal[i] * ray[1] + gY1[i] * s.inv_lam * v.dv;
    gAd[3 * i + 2] = gal[i] * ray[2];
  }
  float gmu_d[3];
  if (!v.parallel) {
    float gd0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gd0[c] = s.Ad[c] * gal[0] + s.Ad[3 + c] * gal[1] + s.Ad[6 + c] * gal[2];
    glam += g_xc * s.d0[0] * v.inv_du + g_yc * s.d0[1] * v.inv_dv;
    gd0[0] += g_xc * s.lam * v.inv_du;
    gd0[1] += g_yc * s.lam * v.inv_dv;
    gd0[2] -= glam * s.lam / s.d0[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) gmu_d[c] = gd0[c];
  } else {
    gmu_d[0] = g_xc * v.inv_du;
    gmu_d[1] = g_yc * v.inv_dv;
    float gt = g_xc * v.dir_d[0] * v.inv_du + g_yc * v.dir_d[1] * v.inv_dv;
    gmu_d[2] = -gt / v.dir_d[2];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) gmu[k] = v.F[k] * gmu_d[0] + v.F[3 + k] * gmu_d[1] + v.F[6 + k] * gmu_d[2];
  // Ad[i][c] = sum_k A[i][k] F[c][k]
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      gA[3 * i + k] = gAd[3 * i] * v.F[k] + gAd[3 * i + 1] * v.F[3 + k] + gAd[3 * i + 2] * v.F[6 + k];
}

// ---- the paper's 2D-Gaussian projection model (Sec. 3.1, Eq. 4) ----------------------------------
// In the detector frame, t = mu' - src; the perspective map to pixels has the Jacobian
//   J = [[a / tz, 0, -a tu / tz^2], [0, b / tz, -b tv / tz^2]],  a = SDD_n / du, b = SDD_n / dv,
// and the projected covariance is Sig2 = J C J^T with C = Sigma' in the detector frame (the EWA covariance
// J W Sigma W^T J^T with its third row and column dropped).  The integration bias factor follows from the
// affine ray-space map (x, y, l = |t|) with Jacobian J3 = [J; t^T / |t|], |det J3| = a b |t| / tz^3:
// the line integral of the ray-space Gaussian over l at fixed (x, y) is
//   rho sqrt(2 pi det(J3 C J3^T) / det Sig2) exp(-Delta^T Sig2^-1 Delta / 2),
// so amp = rho sqrt(2 pi) |det J3| sqrt(det C / det Sig2) = rho sqrt(2 pi) |det J3| / (|det A| sqrt(det Sig2)).
// The record then has N = Sig2^-1, w = 0, kappa = 0 and no per-pixel |X - s| factor.
struct EwaState {
  float t[3], Ai[9], Bm[9], Q0[3], Q1[3], s00, s01, s11, det2, detA, a, b, ell, detJ3, amp, xc, yc;
};

__device__ __forceinline__ bool ewa_core(const ViewC& v, const float mu[3], const float A[9], float rho, EwaState& e) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
    e.t[c] = v.F[3 * c] * mu[0] + v.F[3 * c + 1] * mu[1] + v.F[3 * c + 2] * mu[2] - v.src_d[c];
  const float tz = e.t[2];
  if (!(tz > 0.f)) return false;
  e.detA = inv3(A, e.Ai);  // returns det A; Ai = A^-1, so Sigma' = Ai Ai^T
  if (!(fabsf(e.detA) > 0.f)) return false;
  // Bm = F Ai: Sigma' in the detector frame is C = Bm Bm^T
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      e.Bm[3 * c + k] = v.F[3 * c] * e.Ai[k] + v.F[3 * c + 1] * e.Ai[3 + k] + v.F[3 * c + 2] * e.Ai[6 + k];
  e.a = v.sdd_n * v.inv_du;
  e.b = v.sdd_n * v.inv_dv;
  const float itz = 1.f / tz;
  const float j00 = e.a * itz, j02 = -e.a * e.t[0] * itz * itz, j11 = e.b * itz, j12 = -e.b * e.t[1] * itz * itz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e.Q0[k] = j00 * e.Bm[k] + j02 * e.Bm[6 + k];
    e.Q1[k] = j11 * e.Bm[3 + k] + j12 * e.Bm[6 + k];
  }
  e.s00 = e.Q0[0] * e.Q0[0] + e.Q0[1] * e.Q0[1] + e.Q0[2] * e.Q0[2];
  e.s01 = e.Q0[0] * e.Q1[0] + e.Q0[1] * e.Q1[1] + e.Q0[2] * e.Q1[2];
  e.s11 = e.Q1[0] * e.Q1[0] + e.Q1[1] * e.Q1[1] + e.Q1[2] * e.Q1[2];
  e.det2 = e.s00 * e.s11 - e.s01 * e.s01;
  if (!(e.det2 > 0.f)) return false;
  e.ell = sqrtf(e.t[0] * e.t[0] + e.t[1] * e.t[1] + tz * tz);
  e.detJ3 = e.a * e.b * e.ell * itz * itz * itz;
  e.amp = rho * DIGS_SQRT_2PI * e.detJ3 / (fabsf(e.detA) * sqrtf(e.det2));
  e.xc = v.cx0 + (v.su + v.sdd_n * e.t[0] * itz) * v.inv_du;
  e.yc = v.cy0 + (v.sv + v.sdd_n * e.t[1] * itz) * v.inv_dv;
  return isfinite(e.xc) && isfinite(e.yc) && isfinite(e.amp) && isfinite(e.det2);
}

// Record and pixel box of { Delta : Delta^T Sig2^-1 Delta <= c2 } (half widths sqrt(c2 Sig2_ii)).
__device__ __forceinline__ bool ewa_record(const ViewC& v, const float mu[3], const float A[9], float rho, float c2,
                                           Rec& r) {
  EwaState e;
  if (!ewa_core(v, mu, A, rho, e)) return false;
  const float hx = sqrtf(c2 * e.s00) * 1.0001f + 1e-3f, hy = sqrtf(c2 * e.s11) * 1.0001f + 1e-3f;
  float fx0 = fmaxf(ceilf(e.xc - hx), 0.f), fx1 = fminf(floorf(e.xc + hx), (float)(v.nu - 1));
  float fy0 = fmaxf(ceilf(e.yc - hy), 0.f), fy1 = fminf(floorf(e.yc + hy), (float)(v.nv - 1));
  if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
  const float id = 1.f / e.det2;
  r.xc = e.xc; r.yc = e.yc;
  r.n00 = e.s11 * id; r.n01x2 = -2.f * e.s01 * id; r.n11 = e.s00 * id;
  r.wn0 = 0.f; r.wn1 = 0.f; r.kappa = 0.f; r.amp = e.amp;
  r.bx = (int)fx0 | ((int)fx1 << 16);
  r.by = (int)fy0 | ((int)fy1 << 16);
  r.poly = 1;
  return true;
}

// Adjoint of ewa_core: from dL/d(xc, yc, n00, n01, n11, amp) (n01 the off-diagonal of N = Sig2^-1) to
// dL/dmu (world), dL/dA and dL/drho.
__device__ __forceinline__ void ewa_adjoint(const ViewC& v, const EwaState& e, float rho, float g_xc, float g_yc,
                                            float g_n00, float g_n01, float g_n11, float gamp, float gmu[3],
                                            float gA[9], float& grho) {
  const float id = 1.f / e.det2, ga = gamp * e.amp;  // dL/damp * amp
  grho = gamp * e.amp / rho;
  // N = [[s11, -s01], [-s01, s00]] / det2; amp ~ det2^-1/2
  const float gdet = -(g_n00 * e.s11 - g_n01 * e.s01 + g_n11 * e.s00) * id * id - 0.5f * ga * id;
  const float g00 = g_n11 * id + gdet * e.s11, g11 = g_n00 * id + gdet * e.s00;
  const float g01 = -g_n01 * id - 2.f * gdet * e.s01;
  // Sig2 = Q Q^T
  float gQ0[3], gQ1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gQ0[k] = 2.f * g00 * e.Q0[k] + g01 * e.Q1[k];
    gQ1[k] = 2.f * g11 * e.Q1[k] + g01 * e.Q0[k];
  }
  // Q0 = j00 Bm[0,:] + j02 Bm[2,:], Q1 = j11 Bm[1,:] + j12 Bm[2,:]
  const float tz = e.t[2], itz = 1.f / tz;
  const float j00 = e.a * itz, j02 = -e.a * e.t[0] * itz * itz, j11 = e.b * itz, j12 = -e.b * e.t[1] * itz * itz;
  float gBm[9];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gBm[k] = j00 * gQ0[k];
    gBm[3 + k] = j11 * gQ1[k];
    gBm[6 + k] = j02 * gQ0[k] + j12 * gQ1[k];
  }
  float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gj00 += gQ0[k] * e.Bm[k];
    gj02 += gQ0[k] * e.Bm[6 + k];
    gj11 += gQ1[k] * e.Bm[3 + k];
    gj12 += gQ1[k] * e.Bm[6 + k];
  }
  // t: the Jacobian entries, the projected mean and |det J3| = a b |t| / tz^3
  float gt[3];
  gt[0] = gj02 * (-e.a * itz * itz) + g_xc * e.a * itz + ga * e.t[0] / (e.ell * e.ell);
  gt[1] = gj12 * (-e.b * itz * itz) + g_yc * e.b * itz + ga * e.t[1] / (e.ell * e.ell);
  gt[2] = gj00 * (-e.a * itz * itz) + gj02 * (2.f * e.a * e.t[0] * itz * itz * itz) + gj11 * (-e.b * itz * itz) +
          gj12 * (2.f * e.b * e.t[1] * itz * itz * itz) - g_xc * e.a * e.t[0] * itz * itz -
          g_yc * e.b * e.t[1] * itz * itz + ga * (tz / (e.ell * e.ell) - 3.f * itz);
#pragma unroll
  for (int k = 0; k < 3; ++k) gmu[k] = v.F[k] * gt[0] + v.F[3 + k] * gt[1] + v.F[6 + k] * gt[2];
  // Bm = F Ai  ->  gAi = F^T gBm;  Ai = A^-1  ->  gA = -Ai^T gAi Ai^T;  |det A|^-1 in amp -> -ga Ai^T
  float gAi[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      gAi[3 * i + k] = v.F[i] * gBm[k] + v.F[3 + i] * gBm[3 + k] + v.F[6 + i] * gBm[6 + k];
  float T1[9];  // Ai^T gAi
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      T1[3 * i + k] = e.Ai[i] * gAi[k] + e.Ai[3 + i] * gAi[3 + k] + e.Ai[6 + i] * gAi[6 + k];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      gA[3 * i + k] = -(T1[3 * i] * e.Ai[k * 3] + T1[3 * i + 1] * e.Ai[k * 3 + 1] + T1[3 * i + 2] * e.Ai[k * 3 + 2]) -
                      ga * e.Ai[3 * k + i];
}
