// Low-rank cubic B-spline FFD (Sec. 3.3, Eq. 9-11): value, world-space gradient and the backward pass
// of both, for one point per thread.
#pragma once

#include "digs_common.cuh"

// Uniform cubic B-spline basis at local coordinate u in [0, 1) and its first and second derivatives
// with respect to u (the FFD basis the paper cites for Eq. 10).
__device__ __forceinline__ void bspline4(float u, float B[4]) {
  float v = 1.f - u, u2 = u * u, u3 = u2 * u;
  B[0] = v * v * v * (1.f / 6.f);
  B[1] = (3.f * u3 - 6.f * u2 + 4.f) * (1.f / 6.f);
  B[2] = (-3.f * u3 + 3.f * u2 + 3.f * u + 1.f) * (1.f / 6.f);
  B[3] = u3 * (1.f / 6.f);
}

__device__ __forceinline__ void bspline4_d1(float u, float dB[4]) {
  float v = 1.f - u;
  dB[0] = -0.5f * v * v;
  dB[1] = 1.5f * u * u - 2.f * u;
  dB[2] = -1.5f * u * u + u + 0.5f;
  dB[3] = 0.5f * u * u;
}

__device__ __forceinline__ void bspline4_d2(float u, float d2B[4]) {
  d2B[0] = 1.f - u;
  d2B[1] = 3.f * u - 2.f;
  d2B[2] = 1.f - 3.f * u;
  d2B[3] = u;
}

// Lattice cell of x: floor(p) - 1 is the first of the 4 nodes per axis (Eq. 10), u = p - floor(p).
__device__ __forceinline__ void lattice_cell(const LatticeC& L, const float x[3], int f[3], float u[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float p = (x[a] - L.origin[a]) * L.inv_h[a];
    float fl = floorf(p);
    f[a] = (int)fl - 1;
    u[a] = p - fl;
  }
}

// u_r(x) (U[r][c]) and d u_{r,c} / d x_j (dU[r][3c + j]) for R ranks.  Nodes outside the lattice are
// skipped, i.e. read as zero displacement.
template <int R>
__device__ __forceinline__ void ffd_eval_point(const float* __restrict__ phi, const LatticeC& L, const float x[3],
                                               float U[R][3], float dU[R][9]) {
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
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) U[r][c] = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) dU[r][c] = 0.f;
  }
  const size_t rank_stride = (size_t)L.nx * L.ny * L.nz * 3;
  for (int n3 = 0; n3 < 4; ++n3) {
    int k = f[2] + n3;
    if (k < 0 || k >= L.nz) continue;
    for (int m = 0; m < 4; ++m) {
      int j = f[1] + m;
      if (j < 0 || j >= L.ny) continue;
      float wyz = B[1][m] * B[2][n3], gyz_y = dB[1][m] * B[2][n3], gyz_z = B[1][m] * dB[2][n3];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        int i = f[0] + l;
        if (i < 0 || i >= L.nx) continue;
        float wt = B[0][l] * wyz, gx = dB[0][l] * wyz, gy = B[0][l] * gyz_y, gz = B[0][l] * gyz_z;
        const float* d = phi + (((size_t)k * L.ny + j) * L.nx + i) * 3;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float d0 = __ldg(d + r * rank_stride), d1 = __ldg(d + r * rank_stride + 1), d2 = __ldg(d + r * rank_stride + 2);
          U[r][0] = fmaf(wt, d0, U[r][0]);
          U[r][1] = fmaf(wt, d1, U[r][1]);
          U[r][2] = fmaf(wt, d2, U[r][2]);
          dU[r][0] = fmaf(gx, d0, dU[r][0]); dU[r][1] = fmaf(gy, d0, dU[r][1]); dU[r][2] = fmaf(gz, d0, dU[r][2]);
          dU[r][3] = fmaf(gx, d1, dU[r][3]); dU[r][4] = fmaf(gy, d1, dU[r][4]); dU[r][5] = fmaf(gz, d1, dU[r][5]);
          dU[r][6] = fmaf(gx, d2, dU[r][6]); dU[r][7] = fmaf(gy, d2, dU[r][7]); dU[r][8] = fmaf(gz, d2, dU[r][8]);
        }
      }
    }
  }
}

// Second derivatives d2 u_{r,c} / dx_m dx_j of one rank's field at x (phi_r: that rank's control
// points): H[6 c + s] for s = xx, yy, zz, xy, xz, yz.
__device__ __forceinline__ void ffd_hessian_rank(const float* __restrict__ phi_r, const LatticeC& L, const float x[3],
                                                 float H[18]) {
  int f[3];
  float u[3];
  lattice_cell(L, x, f, u);
  float B[3][4], dB[3][4], d2B[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bspline4(u[a], B[a]);
    bspline4_d1(u[a], dB[a]);
    bspline4_d2(u[a], d2B[a]);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      dB[a][l] *= L.inv_h[a];
      d2B[a][l] *= L.inv_h[a] * L.inv_h[a];
    }
  }
#pragma unroll
  for (int c = 0; c < 18; ++c) H[c] = 0.f;
#pragma unroll
  for (int n3 = 0; n3 < 4; ++n3) {
    int k = f[2] + n3;
    if (k < 0 || k >= L.nz) continue;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int j = f[1] + m;
      if (j < 0 || j >= L.ny) continue;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        int i = f[0] + l;
        if (i < 0 || i >= L.nx) continue;
        const float bx = B[0][l], by = B[1][m], bz = B[2][n3];
        const float dbx = dB[0][l], dby = dB[1][m], dbz = dB[2][n3];
        const float h[6] = {d2B[0][l] * by * bz, bx * d2B[1][m] * bz, bx * by * d2B[2][n3],
                            dbx * dby * bz,      dbx * by * dbz,      bx * dby * dbz};
        const float* d = phi_r + (((size_t)k * L.ny + j) * L.nx + i) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float v = __ldg(d + c);
#pragma unroll
          for (int s = 0; s < 6; ++s) H[6 * c + s] = fmaf(h[s], v, H[6 * c + s]);
        }
      }
    }
  }
}

