// Shared device-side definitions of the DIGS hot path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "digs.h"

#define DIGS_REC_F4 3              // a (projection, Gaussian) record is 3 float4 = 48 bytes
#define DIGS_PARTIAL_F4 3          // the backward's ten sums of a record, padded to 3 float4 = 48 bytes
#define DIGS_FOLD_EPS 1e-6f        // det K at or below this: the deformation folds, drop the Gaussian
#define DIGS_SQRT_2PI 2.5066282746310002f
#define DIGS_LOG2E 1.4426950408889634f

namespace digs {
// Asynchronous global -> shared copies (16 bytes: both addresses 16-byte aligned; 4 bytes: 4-byte
// aligned), their commit groups and the waits for them (per thread).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
}  // namespace digs

// Per-projection geometry, derived on the host in double precision and passed by value.
// The detector frame is (e_u, e_v, n_d) with n_d the unit normal pointing from the source side to the
// detector; every point is handled through its coordinates in that frame so that FP32 never subtracts
// two numbers of the source-distance magnitude (about 1000 mm) to get a millimetre offset.
struct ViewC {
  float F[9];        // rows e_u, e_v, n_d (world -> detector frame)
  float src_d[3];    // source in the detector frame
  float det_d[3];    // detector centre in the detector frame
  float dir_d[3];    // parallel beam: unit ray direction in the detector frame
  float su, sv;      // (src - det_c) . e_u, . e_v
  float sdd_n;       // (det_c - src) . n_d
  float du, dv, inv_du, inv_dv;
  float cx0, cy0;    // pixel coordinates of det_c: (nu - 1) / 2 - off_u, (nv - 1) / 2 - off_v
  int nu, nv;
  int parallel;
  int w_row;         // row of the temporal-weight table used by this projection
  int scan;          // scan whose Gaussians and control points this projection renders
  int ewa;           // 1: the paper's 2D-Gaussian (EWA) projection model instead of the exact line integral
};

struct ViewsParam {
  ViewC v[DIGS_MAX_VIEWS];
};

// Scans sharing one call: scan s owns Gaussians [off[s], off[s+1]); records are laid out
// [projection][nmax]; phi of scan s starts phi_stride floats after that of scan s - 1.
struct ScanTable {
  int S;
  int off[DIGS_MAX_SCANS + 1];
  int nmax;
  long long phi_stride;
};

__device__ __forceinline__ int scan_of(const ScanTable& T, int g) {
  int s = 0;
#pragma unroll
  for (int k = 1; k < DIGS_MAX_SCANS; ++k) s += (k < T.S && g >= T.off[k]) ? 1 : 0;
  return s;
}

struct LatticeC {
  float origin[3];
  float inv_h[3];    // 1 / spacing
  int nx, ny, nz, R;
};

struct GaussPtrs {
  const float* mu0;
  const float* scale;
  const float* quat;
  const float* rho;
  int n;
};

// Record of one (projection, Gaussian) pair after the deformation-informed warp and projection set-up.
// With Delta = (px - xc, py - yc) the pixel offset from the projected mean (in pixels):
//   num = n00 dx^2 + n01x2 dx dy + n11 dy^2,   t = 1 + wn0 dx + wn1 dy,   D = t^2 + kappa num,
//   E = num / D (squared Mahalanobis distance from the ray to the mean),
//   V = amp * L_pix * D^-1/2 * exp(-E / 2) (the whole-line integral; L_pix = |pixel - source| per pixel).
// Words 9 and 10 hold the inclusive pixel box (x0 | x1 << 16, y0 | y1 << 16) outside which E > cutoff^2;
// word 11 is 1 when |D - 1| <= 0.02 over the box (D^-1/2 may then be taken from its binomial series).
struct Rec {
  float xc, yc, n00, n01x2, n11, wn0, wn1, kappa, amp;
  int bx, by, poly;
};

__device__ __forceinline__ Rec load_rec(const float4* r3) {
  float4 a = r3[0], b = r3[1], c = r3[2];
  Rec r;
  r.xc = a.x; r.yc = a.y; r.n00 = a.z; r.n01x2 = a.w;
  r.n11 = b.x; r.wn0 = b.y; r.wn1 = b.z; r.kappa = b.w;
  r.amp = c.x; r.bx = __float_as_int(c.y); r.by = __float_as_int(c.z); r.poly = __float_as_int(c.w);
  return r;
}

__device__ __forceinline__ void store_rec(float4* r3, const Rec& r) {
  r3[0] = make_float4(r.xc, r.yc, r.n00, r.n01x2);
  r3[1] = make_float4(r.n11, r.wn0, r.wn1, r.kappa);
  r3[2] = make_float4(r.amp, __int_as_float(r.bx), __int_as_float(r.by), __int_as_float(r.poly));
}

// |pixel centre - source| for pixel (px, py) (cone beam, exact model); 1 for parallel beams and for the
// 2D-Gaussian model, whose amplitude already holds the whole line integral.
__device__ __forceinline__ float pixel_ray_length(const ViewC& v, float px, float py) {
  if (v.parallel || v.ewa) return 1.f;
  float a = (px - v.cx0) * v.du - v.su;
  float b = (py - v.cy0) * v.dv - v.sv;
  return sqrtf(fmaf(a, a, fmaf(b, b, v.sdd_n * v.sdd_n)));
}

__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
