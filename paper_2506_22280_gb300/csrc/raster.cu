// Tile rasteriser of the X-ray transform (Sec. 3.1, Eq. 1, 3-4) and its backward pass.
//
// Per pixel, with (dx, dy) its offset from the projected mean:
//   num = n00 dx^2 + n01x2 dx dy + n11 dy^2,  t = 1 + wn0 dx + wn1 dy,  D = t^2 + kappa num,  E = num / D,
// and the pixel takes V = amp |X - s| D^-1/2 exp(-E/2) when E <= cutoff^2.  The constant k = -log2(e)/2
// is folded into num, so that k E is directly the argument of the SFU's exp2; D^-1/2 is the SFU's
// reciprocal square root.  Pixels are taken two at a time in packed FP32x2 arithmetic
// (fma/mul/add.rn.f32x2).
//
// Forward: one CTA per (projection, tile) and one warp per 8 x 8 block of the tile; each lane owns two
// pixels of the block and keeps their sums in registers.  Every warp walks the tile's sorted Gaussian
// list in batches of 32 records staged by cp.async, keeps the Gaussians whose cutoff ellipse meets its
// block and sweeps them eight at a time, summed in list order: no canvas, no atomics, deterministic sums.
// An entry carries its quadratic form scaled by 1/|amp|^2 (and t by 1/|amp|), so that the reciprocal
// square root of the scaled D is |amp| D^-1/2; the accumulating FMA applies the sign of amp.  CTAs start
// in order of decreasing list length.
//
// Backward: needs no tile lists.  One half-warp per (projection, Gaussian) record (the two records of a
// warp of similar box size, paired by k_bwd_pairing) sweeps the record's pixel box in 16-column slices,
// reading g = dL/dI * |X - s| from the projection-sized image (L1/L2 resident).  Narrow slices (w <= 8):
// lane l owns column (l mod w), starts at row (l div w) and takes the row pair (r, r + s), s = 16 div w,
// stepping 2s rows; wider slices: the column pair (c, c + ceil(w/2)) of row (l div ceil(w/2)), stepping
// s = 16 div ceil(w/2) rows.  Each lane accumulates seven sums per pixel of its pair and turns them into
// the ten sufficient statistics of the record gradient; the half-warp reduces them with an 11-shuffle
// recursive halving and ten lanes write them to the record's slot (no atomics).  A CTA sweeps four units
// of 16 records in turn, each unit's records and tile counts copied to shared memory by cp.async while
// the unit before it is swept.
//
// Loss: per-warp partials of the squared residuals from the forward, summed in two fixed-order levels.
#include <algorithm>

#include "digs_internal.h"

namespace digs {

constexpr float kNegHalfLog2e = -0.5f * DIGS_LOG2E;


// ---- packed FP32x2: the two pixels of a lane's pair in one register pair ------------------------
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2 f2_dup(float x) { return f2_pack(x, x); }
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// The SFU's 2^x and 1/sqrt(x) (PTX ex2.approx / rsqrt.approx, flushing subnormals: the arguments here
// are in [-9, 0] and near 1).
__device__ __forceinline__ float sfu_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sfu_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ f2 f2_exp2(f2 x) {
  float a, b;
  f2_unpack(x, a, b);
  return f2_pack(sfu_exp2(a), sfu_exp2(b));
}
__device__ __forceinline__ f2 f2_rsqrt(f2 x) {
  float a, b;
  f2_unpack(x, a, b);
  return f2_pack(sfu_rsqrt(a), sfu_rsqrt(b));
}

// ---- lane layouts (forward and backward) ---------------------------------------------------------

// Lane layout of a box slice w <= LPR pixels wide for a group of LPR lanes (16 or 32) sharing one
// record, per w: cw | s << 6 | m << 12, where cw is the number of lane columns, s the rows covered per
// pass and m = ceil(1024 / cw), so that (l * m) >> 10 = l / cw exactly for l < 32 (cw <= 16).
// w <= LPR/2: lane l takes column l mod w and the row pair (r, r + s), s = LPR div w, stepping 2s rows.
// LPR/2 < w <= LPR: the column pair (c, c + ceil(w/2)), stepping s = LPR div ceil(w/2) rows.
template <int LPR>
struct LaneTable {
  int v[LPR + 1];
  constexpr LaneTable() : v() {
    for (int w = 1; w <= LPR; ++w) {
      const int cw = w <= LPR / 2 ? w : (w + 1) / 2;
      v[w] = cw | ((LPR / cw) << 6) | (((1024 + cw - 1) / cw) << 12);
    }
  }
};
__constant__ LaneTable<16> kLanes16 = LaneTable<16>();
__constant__ LaneTable<32> kLanes32 = LaneTable<32>();

struct HalfLanes {
  int c, r0, pdx, pdy, ystep;
  bool active, col2;
};
template <int LPR>
__device__ __forceinline__ HalfLanes group_lanes(int w, int h, int hl) {
  const int t = LPR == 16 ? kLanes16.v[w] : kLanes32.v[w];
  const int cw = t & 63, s = (t >> 6) & 63, m = t >> 12;
  const int q = (hl * m) >> 10;
  const bool rows = w <= LPR / 2;
  HalfLanes L;
  L.c = hl - q * cw;
  L.r0 = q;
  L.pdx = rows ? 0 : cw;
  L.pdy = rows ? s : 0;
  L.ystep = rows ? 2 * s : s;
  L.active = q < s && q < h;
  L.col2 = L.c + L.pdx < w;
  return L;
}

// ---- forward ------------------------------------------------------------------------------------

// One CTA per (projection, tile), launched in the order `order` gives; one warp per 8 x 8 block of the tile.  Lane l owns the pixels
// (l mod 8, l div 8) and (l mod 8, l div 8 + 4) of its block and keeps their sums in a register pair.
template <int TS>
struct FwdCfg {
  static constexpr int blocks_x = TS / 8;
  static constexpr int warps = blocks_x * blocks_x;
  static constexpr int threads = 32 * warps;
  static constexpr int batch = 32;                              // records a warp stages at a time
  static constexpr int raw_f4 = batch * DIGS_REC_F4;            // staged records
  static constexpr int ent_f4 = batch * 3;                      // derived entries
  static constexpr size_t smem = (size_t)warps * (raw_f4 + ent_f4) * sizeof(float4);
};

// A staged record -> the entry the pixel loop reads:
//   (k n00 / sg^2, k n01x2 / sg^2, k n11 / sg^2, wn0 / sg), (wn1 / sg, kappa / k, amp / sg, -xc), (-yc, 1 / sg, 0, 0)
// with k = -log2(e) / 2, so that the loop forms the exp2 argument k E = k num / D directly, and
// sg = |amp| (1 when |amp| lies outside [2^-40, 2^40]): num and t scaled by 1 / sg^2 and 1 / sg scale D
// by 1 / sg^2 and leave E unchanged, so the SFU's rsqrt of the scaled D is sg D^-1/2 and the amplitude
// costs no multiply in the loop (amp / sg, i.e. the sign of amp, is applied by the accumulating FMA).
__device__ __forceinline__ void derive_entry(const float4* raw, float4* ent) {
  const float4 a = raw[0], b = raw[1], c = raw[2];
  const float mag = fabsf(c.x);
  const bool fold = mag >= 0x1p-40f && mag <= 0x1p40f;
  const float s1 = fold ? __frcp_rn(mag) : 1.f, s2 = s1 * s1;
  const float sgn = fold ? copysignf(1.f, c.x) : c.x;
  ent[0] = make_float4(kNegHalfLog2e * a.z * s2, kNegHalfLog2e * a.w * s2, kNegHalfLog2e * b.x * s2, b.y * s1);
  ent[1] = make_float4(b.z * s1, b.w * (1.f / kNegHalfLog2e), sgn, -a.x);
  ent[2] = make_float4(-a.y, s1, 0.f, 0.f);
}

// Whether the pixel rectangle [x0, x1] x [y0, y1] (a block's part of the record's box) can hold a pixel
// with E <= c2: E = num / D with D <= Dmax = (1 + tau)^2 / (1 - c2 kappa) over the box (|t - 1| <= tau,
// kappa num <= c2 kappa D), so no pixel qualifies when min over the rectangle of the quadratic form num
// exceeds c2 Dmax.  The minimum of a positive definite form over a rectangle not holding its centre lies
// on an edge, where it is a clamped one-dimensional minimum.  Conservative (small relative margin); a
// culled block's entries would only have added zeros, so sums are unchanged.
__device__ __forceinline__ bool ellipse_meets(const float4* r3, int x0, int x1, int y0, int y1, float c2_const) {
  const float4 a = r3[0], b = r3[1], c = r3[2];
  const float xc = a.x, yc = a.y, n00 = a.z, n01 = 0.5f * a.w, n11 = b.x;
  const float X0 = (float)x0 - xc, X1 = (float)x1 - xc, Y0 = (float)y0 - yc, Y1 = (float)y1 - yc;
  if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return true;
  const int bx = __float_as_int(c.y), by = __float_as_int(c.z);
  const float mdx = fmaxf(fabsf((float)(bx & 0xffff) - xc), fabsf((float)(bx >> 16) - xc));
  const float mdy = fmaxf(fabsf((float)(by & 0xffff) - yc), fabsf((float)(by >> 16) - yc));
  const float tau = fabsf(b.y) * mdx + fabsf(b.z) * mdy;
  const float ck = 1.f - c2_const * b.w;  // > 0: the source lies outside the cutoff ellipsoid
  if (!(ck > 0.f)) return true;
  // fast (approximate) divisions: they move the clamped minimisers by a few ulps, far inside the margin
  const float lim = __fdividef(c2_const * (1.f + tau) * (1.f + tau), ck) * 1.001f + 1e-4f;
  const float s11 = __fdividef(-n01, n11), s00 = __fdividef(-n01, n00);
  auto q = [&](float dx, float dy) { return dy * (n11 * dy + 2.f * n01 * dx) + n00 * dx * dx; };
  auto edge_x = [&](float dx) {  // min over dy in [Y0, Y1] at fixed dx
    const float dy = fminf(fmaxf(s11 * dx, Y0), Y1);
    return q(dx, dy);
  };
  auto edge_y = [&](float dy) {
    const float dx = fminf(fmaxf(s00 * dy, X0), X1);
    return q(dx, dy);
  };
  const float m = fminf(fminf(edge_x(X0), edge_x(X1)), fminf(edge_y(Y0), edge_y(Y1)));
  return !(m > lim);
}

__device__ __forceinline__ f2 f2_lo(const float4& v) { return f2_pack(v.x, v.y); }
__device__ __forceinline__ f2 f2_hi(const float4& v) { return f2_pack(v.z, v.w); }

// V / (|X - s| amp / sg) of one entry at the lane's two pixels (XX, YY), zero outside the cutoff
// (k E < c2k); *sgn = amp / sg, the factor the caller accumulates it with.
template <bool COUNT>
__device__ __forceinline__ f2 fwd_pair(const float4* en, float xx, f2 YY, float c2k, unsigned& n_cut, float& sgn) {
  const float4 q0 = en[0], q1 = en[1], q2 = en[2];
  // the lane's two pixels share their column: the dx terms are scalars
  const float dx = xx + q1.w;
  const float aq = q0.x * dx * dx, bq = q0.y * dx, t0 = fmaf(q0.w, dx, q2.y);
  const f2 DY = f2_add(YY, f2_dup(q2.x));
  const f2 NUM = f2_fma(DY, f2_fma(f2_dup(q0.z), DY, f2_dup(bq)), f2_dup(aq));  // k num / sg^2
  const f2 T = f2_fma(f2_dup(q1.x), DY, f2_dup(t0));                             // t / sg
  const f2 D = f2_fma(T, T, f2_mul(f2_dup(q1.y), NUM));                          // D / sg^2
  const f2 RS = f2_rsqrt(D);                                                      // sg D^-1/2
  const f2 ARG = f2_mul(NUM, f2_mul(RS, RS));                                     // k E
  const f2 VAL = f2_mul(RS, f2_exp2(ARG));
  float aa, ab, va, vb;
  f2_unpack(ARG, aa, ab);
  f2_unpack(VAL, va, vb);
  const bool ia = aa >= c2k, ib = ab >= c2k;
  if (COUNT) n_cut += (unsigned)ia + (unsigned)ib;
  sgn = q1.z;
  return f2_pack(ia ? va : 0.f, ib ? vb : 0.f);
}

// Each warp walks the tile's whole sorted list in batches of 32: lane l copies record l of the batch
// into shared memory (cp.async), tests its box against the warp's block and, if they meet, writes the
// entry to the slot given by the number of meeting lanes below it (so the meeting entries lie packed,
// in list order); the next batch's copies are then issued and the warp sweeps the packed entries in
// order (so the sums are deterministic).  No canvas, no atomics, no CTA barrier.
template <int TS, bool COUNT>
__global__ void __launch_bounds__(FwdCfg<TS>::threads) k_raster_fwd(
    const float4* __restrict__ grec, const uint32_t* __restrict__ srid, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ order, const __grid_constant__ ViewsParam views, int tiles_x, int T, int nu, int nv,
    float c2, float* __restrict__ proj, const float* __restrict__ meas, float* __restrict__ dldi,
    float* __restrict__ loss_part, float inv_count, unsigned long long* __restrict__ counters) {
  using C = FwdCfg<TS>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* raw = (float4*)smem + (size_t)warp * (C::raw_f4 + C::ent_f4);
  float4* ent = raw + C::raw_f4;
  const uint32_t bt = order[blockIdx.x];  // heaviest (projection, tile) lists first
  const int b = (int)(bt / (uint32_t)T), tile = (int)(bt % (uint32_t)T);
  const int qx = (tile % tiles_x) * TS + (warp % C::blocks_x) * 8, qy = (tile / tiles_x) * TS + (warp / C::blocks_x) * 8;
  const int px = qx + (lane & 7), py = qy + (lane >> 3);  // the lane's pixels: (px, py) and (px, py + 4)
  const float XX = (float)px;
  const f2 YY = f2_pack((float)py, (float)(py + 4));
  const uint2 rg = ranges[(size_t)b * T + tile];
  const float c2k = c2 * kNegHalfLog2e;
  f2 ACC = f2_dup(0.f);
  unsigned n_box = 0, n_cut = 0;
  auto issue = [&](uint32_t k0) {
    const uint32_t k = k0 + lane;
    if (k < rg.y) {
      const float4* src = grec + (size_t)srid[k] * DIGS_REC_F4;
#pragma unroll
      for (int q = 0; q < DIGS_REC_F4; ++q) cp_async16(raw + lane * DIGS_REC_F4 + q, src + q);
    }
    cp_async_commit();
  };
  if (rg.x < rg.y) issue(rg.x);
  for (uint32_t k0 = rg.x; k0 < rg.y; k0 += C::batch) {
    cp_async_wait_all();
    bool meets = false;
    if (k0 + lane < rg.y) {
      const float4* r3 = raw + lane * DIGS_REC_F4;
      const float4 c = r3[2];
      const int bx = __float_as_int(c.y), by = __float_as_int(c.z);
      const int x0 = max(bx & 0xffff, qx), x1 = min(bx >> 16, qx + 7);
      const int y0 = max(by & 0xffff, qy), y1 = min(by >> 16, qy + 7);
      meets = x0 <= x1 && y0 <= y1;
      if (COUNT && meets) n_box += (unsigned)((x1 - x0 + 1) * (y1 - y0 + 1));
      meets = meets && ellipse_meets(r3, x0, x1, y0, y1, c2);
    }
    // the meeting entries, compacted in list order: lane -> slot popc(mask below the lane)
    const unsigned mask = __ballot_sync(0xffffffffu, meets);
    if (meets) derive_entry(raw + lane * DIGS_REC_F4, ent + __popc(mask & ((1u << lane) - 1u)) * 3);
    __syncwarp();
    issue(k0 + C::batch);  // lands while this batch is swept
    const int cnt = __popc(mask);
    int e = 0;
    // n entries from e: all evaluated (independent dependency chains), then accumulated in list order
    auto sweep = [&](int n) {
      f2 v[8];
      float sg[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < n) v[k] = fwd_pair<COUNT>(ent + (e + k) * 3, XX, YY, c2k, n_cut, sg[k]);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < n) ACC = f2_fma(f2_dup(sg[k]), v[k], ACC);
    };
#pragma unroll 1
    for (; e + 7 < cnt; e += 8) sweep(8);  // eight entries per step
    if (e + 3 < cnt) { sweep(4); e += 4; }
    if (e + 1 < cnt) { sweep(2); e += 2; }
    if (e < cnt) sweep(1);
    __syncwarp();
  }
  cp_async_wait_all();  // the last (empty) group
  const ViewC& v = views.v[b];
  float s0, s1;
  f2_unpack(ACC, s0, s1);
  float lsum = 0.f;
  auto emit = [&](int y, float sum) {
    if (px < nu && y < nv) {
      const float lp = pixel_ray_length(v, (float)px, (float)y);
      const float I = sum * lp;
      const size_t idx = ((size_t)b * nv + y) * nu + px;
      if (proj) proj[idx] = I;
      if (meas) {
        const float res = I - meas[idx];
        lsum = fmaf(res, res, lsum);
        if (dldi) dldi[idx] = 2.f * res * inv_count * lp;  // dL/dI * |X - s|, what the backward consumes
      }
    }
  };
  emit(py, s0);
  emit(py + 4, s1);
  if (COUNT) {
    unsigned c = n_cut, nb = n_box;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c += __shfl_xor_sync(0xffffffffu, c, o);
      nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if (lane == 0 && (nb | c)) {
      atomicAdd(counters, (unsigned long long)nb);
      atomicAdd(counters + 1, (unsigned long long)c);
    }
  }
  if (loss_part) {  // one partial per warp: no CTA barrier
    lsum = warp_sum(lsum);
    if (lane == 0) loss_part[((size_t)b * T + tile) * C::warps + warp] = lsum;
  }
}

// ---- backward: one half-warp per (projection, Gaussian) record, over the record's whole pixel box ----

constexpr int kBwdThreads = 256;
constexpr int kBwdRounds = 4;  // record units per backward CTA

// Adds the lane's share of the ten record-gradient sums, all but the first divided by amp / 2:
// sum g V/amp; sum dL/dnum (dx^2, dx dy, dy^2); sum dL/dnum (dx, dy); sum dL/dt (1, dx, dy);
// sum dL/dkappa.  gp points at g = dL/dI * |X - s| of the lane's first pixel in the projection image
// (row pitch nu); (dx1, dy1) is that pixel's offset from the projected mean.
//
// Per pixel, with A = (g V / amp) / D and B = A (E - 1): dL/dnum = kappa B - A, dL/dt / 2 = B t and
// dL/dkappa = B num.  A lane's pixel keeps its column, so t = t0 + wn1 dy and num = a + b dy + n11 dy^2
// with column constants t0, a, b: every sum above is a combination of the six dy-moments
// sum A dy^j and sum B dy^j (j = 0, 1, 2), which are all the loop accumulates besides sum g V / amp.
__device__ __forceinline__ void bwd_box_pixels(const Rec& R0, const HalfLanes& B, int h, float dx1, float dy1,
                                               const float* __restrict__ gp, int nu, float c2, float Sv[10]) {
  // k = -log2(e) / 2 is folded into the quadratic form: NUM = k num, ARG = k E (the exp2 argument)
  const float dx2 = dx1 + (float)B.pdx;
  const f2 DX = f2_pack(dx1, dx2);
  const f2 AQ = f2_mul(f2_mul(f2_dup(kNegHalfLog2e * R0.n00), DX), DX);
  const f2 BQ = f2_mul(f2_dup(kNegHalfLog2e * R0.n01x2), DX);
  const f2 T0 = f2_fma(f2_dup(R0.wn0), DX, f2_dup(1.f));
  const f2 N11 = f2_dup(kNegHalfLog2e * R0.n11), WN1 = f2_dup(R0.wn1);
  const f2 KAPK = f2_dup(R0.kappa * (1.f / kNegHalfLog2e));
  const f2 IK = f2_dup(1.f / kNegHalfLog2e), MONE = f2_dup(-1.f), STEP = f2_dup((float)B.ystep);
  const f2 C2K = f2_dup(c2 * kNegHalfLog2e);
  const int pstep = B.ystep * nu, d2 = B.pdy * nu + B.pdx, hb = B.col2 ? h - B.pdy : 0;
  f2 DY = f2_pack(dy1, dy1 + (float)B.pdy);
  f2 S0 = f2_dup(0.f), A0 = S0, A1 = S0, A2 = S0, B0 = S0, B1 = S0, B2 = S0;
  for (int r = B.r0; r < h; r += B.ystep, DY = f2_add(DY, STEP), gp += pstep) {
    f2 NUM = f2_fma(DY, f2_fma(N11, DY, BQ), AQ);
    f2 T = f2_fma(WN1, DY, T0);
    f2 D = f2_fma(T, T, f2_mul(KAPK, NUM));
    // E <= cutoff^2 taken as num <= c2 D (D > 0), i.e. k num >= k c2 D: known before the SFU work, so
    // the two loads of dL/dI are in flight while it runs
    f2 LIM = f2_mul(C2K, D);
    float na, nb, la, lb;
    f2_unpack(NUM, na, nb);
    f2_unpack(LIM, la, lb);
    const float ga = (na >= la) ? __ldg(gp) : 0.f;
    const float gb = (r < hb && nb >= lb) ? __ldg(gp + d2) : 0.f;  // partner in the box
    f2 RS = f2_rsqrt(D);
    f2 INVD = f2_mul(RS, RS);
    f2 ARG = f2_mul(NUM, INVD);
    f2 BV = f2_mul(RS, f2_exp2(ARG));                      // V / amp
    f2 GA = f2_mul(f2_pack(ga, gb), BV);                  // g V / amp
    S0 = f2_add(S0, GA);
    f2 AL = f2_mul(GA, INVD);                               // A = (dL/dV V / (2 D)) / (amp / 2)
    f2 AE = f2_mul(AL, f2_fma(ARG, IK, MONE));              // B = A (E - 1)
    f2 ALD = f2_mul(AL, DY), AED = f2_mul(AE, DY);
    A0 = f2_add(A0, AL);
    A1 = f2_add(A1, ALD);
    A2 = f2_fma(ALD, DY, A2);
    B0 = f2_add(B0, AE);
    B1 = f2_add(B1, AED);
    B2 = f2_fma(AED, DY, B2);
  }
  // per pixel of the pair: the dy-moments of dL/dnum, dL/dt and dL/dkappa from those of A and B, then
  // the dx-moments from the pixel's column
  float s0[2], a0[2], a1[2], a2[2], b0[2], b1[2], b2[2], aq[2], bq[2], t0[2];
  f2_unpack(S0, s0[0], s0[1]);
  f2_unpack(A0, a0[0], a0[1]);
  f2_unpack(A1, a1[0], a1[1]);
  f2_unpack(A2, a2[0], a2[1]);
  f2_unpack(B0, b0[0], b0[1]);
  f2_unpack(B1, b1[0], b1[1]);
  f2_unpack(B2, b2[0], b2[1]);
  f2_unpack(AQ, aq[0], aq[1]);
  f2_unpack(BQ, bq[0], bq[1]);
  f2_unpack(T0, t0[0], t0[1]);
  const float kap = R0.kappa, wn1 = R0.wn1, n11k = kNegHalfLog2e * R0.n11;
  const float dxs[2] = {dx1, dx2};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float dx = dxs[j];
    const float g0 = fmaf(kap, b0[j], -a0[j]), g1 = fmaf(kap, b1[j], -a1[j]), g2 = fmaf(kap, b2[j], -a2[j]);
    const float th0 = fmaf(t0[j], b0[j], wn1 * b1[j]), th1 = fmaf(t0[j], b1[j], wn1 * b2[j]);
    const float gk = fmaf(aq[j], b0[j], fmaf(bq[j], b1[j], n11k * b2[j]));
    Sv[0] += s0[j];
    Sv[1] += dx * dx * g0;
    Sv[2] += dx * g1;
    Sv[3] += g2;
    Sv[4] += dx * g0;
    Sv[5] += g1;
    Sv[6] += 2.f * th0;
    Sv[7] += 2.f * dx * th0;
    Sv[8] += 2.f * th1;
    Sv[9] += gk * (1.f / kNegHalfLog2e);
  }
}

// Sum ten per-lane values over each group of LPR lanes and store them to out[0..9]: first over each
// half-warp (lanes hl = 0..15), then, for LPR = 32, across the two halves.
// Recursive halving over an uneven split, 5 + 3 + 2 + 1 shuffles: after the xor-8 exchange a lane
// holds five values (0-4 or 5-9), after xor-4 three of those five (local 0-2, or 3-4 plus a pad),
// after xor-2 two, after xor-1 one, the value 5 b3 + 3 b2 + 2 b1 + b0 (b_k = bit k of hl) when that
// lies inside its group of five.
template <int LPR>
__device__ __forceinline__ void group_reduce_store10(const float v[10], float* out, int hl, bool store) {
  const unsigned full = 0xffffffffu;
  float a[5];
  {
    const bool hi = (hl & 8) != 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const float keep = hi ? v[5 + j] : v[j], send = hi ? v[j] : v[5 + j];
      a[j] = keep + __shfl_xor_sync(full, send, 8);
    }
  }
  float b0, b1, b2;
  {
    const bool hi = (hl & 4) != 0;
    const float k0 = hi ? a[3] : a[0], k1 = hi ? a[4] : a[1], k2 = hi ? 0.f : a[2];
    const float s0 = hi ? a[0] : a[3], s1 = hi ? a[1] : a[4], s2 = hi ? a[2] : 0.f;
    b0 = k0 + __shfl_xor_sync(full, s0, 4);
    b1 = k1 + __shfl_xor_sync(full, s1, 4);
    b2 = k2 + __shfl_xor_sync(full, s2, 4);
  }
  float c0, c1;
  {
    const bool hi = (hl & 2) != 0;
    const float k0 = hi ? b2 : b0, k1 = hi ? 0.f : b1;
    const float s0 = hi ? b0 : b2, s1 = hi ? b1 : 0.f;
    c0 = k0 + __shfl_xor_sync(full, s0, 2);
    c1 = k1 + __shfl_xor_sync(full, s1, 2);
  }
  const bool hi = (hl & 1) != 0;
  float d = (hi ? c1 : c0) + __shfl_xor_sync(full, hi ? c0 : c1, 1);
  if (LPR == 32) d += __shfl_xor_sync(full, d, 16);
  const int bit2 = (hl >> 2) & 1;
  const int local = 3 * bit2 + 2 * ((hl >> 1) & 1) + (hl & 1);
  if (store && (LPR == 16 || (threadIdx.x & 16) == 0) && local < (bit2 ? 5 : 3)) out[((hl & 8) ? 5 : 0) + local] = d;
}

// The two records of a backward warp are swept in lockstep, so the warp takes as many passes as the
// longer of the two.  Each warp here ranks a group of 32 consecutive records of one projection by their
// sweep cost (box pixels / 32, written by the set-up: the pass count up to the lane layout's rounding;
// stable: ties in index order; bit-sliced ballots over a 9-bit key, records past n last) and writes
// the record of each rank, so that the backward pairs records of adjacent ranks.
// Grid: (ceil(G / 8), P) with G = ceil(n / 32) groups per projection; 256 threads.
__global__ void __launch_bounds__(256) k_bwd_pairing(const uint8_t* __restrict__ cost, const uint32_t* __restrict__ counts,
                                                     int N, int G, uint8_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const int g = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (g >= G) return;  // whole warps
  const int b = blockIdx.y;
  const int n = g * 32 + lane;
  unsigned key = 511u;
  if (n < N) {
    const size_t i = (size_t)b * N + n;
    key = counts[i] != 0u ? (unsigned)cost[i] : 0u;  // padding records of smaller scans have no tiles
  }
  unsigned lt = 0u, eq = 0xffffffffu;  // lanes with a smaller key; lanes whose key agrees so far
#pragma unroll
  for (int bit = 8; bit >= 0; --bit) {
    const unsigned one = (key >> bit) & 1u;
    const unsigned m = __ballot_sync(0xffffffffu, one);
    if (one) {
      lt |= eq & ~m;
      eq &= m;
    } else {
      eq &= ~m;
    }
  }
  const int rank = __popc(lt) + __popc(eq & ((1u << lane) - 1u));
  perm[((size_t)b * G + g) * 32 + rank] = (uint8_t)lane;
}

// One group of LPR lanes (16: two records per warp, 32: one) per (projection, Gaussian) record: the ten
// sums over every pixel of the record's box, reduced over the group and written to grec[record] (12
// floats, the last two unused).  Records whose Gaussian was culled get zeros.
// Each CTA takes `rounds` consecutive units of 256 / LPR records (unit u of projection b: for LPR = 16
// ranks 16 (u mod 2) .. + 15 of record group u / 2 in k_bwd_pairing's order, else records 8u .. 8u + 7).
// A group's record and its tile count go to shared memory by cp.async two units ahead (double buffer;
// the unit after that has its record index loaded while the current one is swept), so that only a CTA's
// first unit waits for them.
// Grid: (ceil(units / rounds), P), units = ceil(N / (256 / LPR)).
template <int LPR>
__global__ void __launch_bounds__(kBwdThreads, 4) k_raster_bwd(const float4* __restrict__ rec,
                                                                const uint32_t* __restrict__ counts, int N, int nu,
                                                                int nv, const float* __restrict__ gpix, float c2,
                                                                const uint8_t* __restrict__ perm,
                                                                float* __restrict__ grec, int rounds) {
  constexpr int kRecords = kBwdThreads / LPR;  // records per unit
  __shared__ __align__(16) float4 sbuf[2][kRecords][DIGS_REC_F4 + 1];  // record, then its tile count
  const int hl = threadIdx.x & (LPR - 1);
  const int b = blockIdx.y;
  const int slot = (int)(threadIdx.x / LPR);
  const int units = (N + kRecords - 1) / kRecords;
  const int G = (N + 31) >> 5;
  const int u0 = blockIdx.x * rounds;
  auto record_of = [&](int u) -> int {  // this group's record in unit u (N: none)
    if (u >= units || u - u0 >= rounds) return N;
    if (LPR == 16) {  // unit pairs share a group of 32 records, taken in the order of k_bwd_pairing
      const int g = u >> 1;
      return g * 32 + perm[((size_t)b * G + g) * 32 + (u & 1) * 16 + slot];
    }
    return u * kRecords + slot;
  };
  auto fetch = [&](int n, int buf) {  // one commit group per call and thread, empty or not
    if (n < N && hl <= DIGS_REC_F4) {
      const size_t i = (size_t)b * N + n;
      if (hl < DIGS_REC_F4)
        cp_async16(&sbuf[buf][slot][hl], rec + i * DIGS_REC_F4 + hl);
      else
        cp_async4(&sbuf[buf][slot][DIGS_REC_F4], counts + i);
    }
    cp_async_commit();
  };
  int n_cur = record_of(u0), n_next = record_of(u0 + 1);
  fetch(n_cur, 0);
  fetch(n_next, 1);
  const float* gimg = gpix + (size_t)b * nv * nu;
  for (int r = 0; r < rounds; ++r) {
    const int n_after = record_of(u0 + r + 2);  // in flight while this unit is swept
    const int buf = r & 1;
    cp_async_wait_but_one();  // this unit's copies have landed (the next unit's may still be in flight)
    __syncwarp();
    const bool valid = n_cur < N;
    float Sv[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid && __float_as_uint(sbuf[buf][slot][DIGS_REC_F4].x) != 0u) {
      const Rec R0 = load_rec(&sbuf[buf][slot][0]);
      const int x0 = R0.bx & 0xffff, x1 = R0.bx >> 16, y0 = R0.by & 0xffff, y1 = R0.by >> 16;
      const int w = x1 - x0 + 1, h = y1 - y0 + 1;
      for (int cx = 0; cx < w; cx += LPR) {  // boxes wider than LPR pixels: LPR-column slices
        const HalfLanes B = group_lanes<LPR>(min(LPR, w - cx), h, hl);
        if (B.active) {
          const int px = x0 + cx + B.c, py = y0 + B.r0;
          const float* gp = gimg + (size_t)py * nu + px;
          bwd_box_pixels(R0, B, h, (float)px - R0.xc, (float)py - R0.yc, gp, nu, c2, Sv);
        }
      }
      const float amph = 0.5f * R0.amp;
#pragma unroll
      for (int q = 1; q < 10; ++q) Sv[q] *= amph;
    }
    group_reduce_store10<LPR>(Sv, grec + ((size_t)b * N + (valid ? n_cur : 0)) * (DIGS_PARTIAL_F4 * 4),
                              threadIdx.x & 15, valid);
    __syncwarp();  // every lane has read this buffer before it is refilled
    fetch(n_after, buf);
    n_cur = n_next;
    n_next = n_after;
  }
  cp_async_wait_all();
}

// g = dL/dI * |X - s| for every pixel (the per-pixel factor of the line integral, applied once).
__global__ void __launch_bounds__(256) k_gpix(const float* __restrict__ grad_proj, const __grid_constant__ ViewsParam views,
                                              int nu, int nv, float* __restrict__ gpix) {
  const int b = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nu * nv) return;
  const size_t idx = (size_t)b * nu * nv + p;
  gpix[idx] = grad_proj[idx] * pixel_ray_length(views.v[b], (float)(p % nu), (float)(p / nu));
}

template <int TS>
static cudaError_t fwd_launch(const Workspace& ws, const ViewsParam& views, float c2, float* proj, const float* meas,
                              float* dldi, float inv_count, bool count, cudaStream_t st) {
  using C = FwdCfg<TS>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_raster_fwd<TS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    cudaFuncSetAttribute(k_raster_fwd<TS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    configured = true;
  }
  const unsigned grid = (unsigned)ws.T * (unsigned)ws.P;
  float* lp = meas ? ws.loss_part : nullptr;
  if (count)
    k_raster_fwd<TS, true><<<grid, C::threads, C::smem, st>>>(ws.rec, ws.srid, ws.ranges, ws.order, views, ws.tiles_x,
                                                              ws.T, ws.nu, ws.nv, c2, proj, meas, dldi, lp, inv_count,
                                                              ws.counters);
  else
    k_raster_fwd<TS, false><<<grid, C::threads, C::smem, st>>>(ws.rec, ws.srid, ws.ranges, ws.order, views,
                                                               ws.tiles_x, ws.T, ws.nu, ws.nv, c2, proj, meas, dldi,
                                                               lp, inv_count, ws.counters);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_raster_fwd(const Workspace& ws, const ViewsParam& views, float c2, float* proj, const float* meas,
                              float* dldi, float inv_count, cudaStream_t st) {
  if (ws.P <= 0) return cudaSuccess;
  const bool count = meas == nullptr;  // pair statistics are gathered by plain projections only
  switch (ws.tile) {
    case 8: return fwd_launch<8>(ws, views, c2, proj, meas, dldi, inv_count, count, st);
    case 16: return fwd_launch<16>(ws, views, c2, proj, meas, dldi, inv_count, count, st);
    case 32: return fwd_launch<32>(ws, views, c2, proj, meas, dldi, inv_count, count, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_raster_bwd(const Workspace& ws, const ViewsParam& views, float c2, const float* grad_proj,
                              cudaStream_t st) {
  if (ws.P <= 0 || ws.n <= 0) return cudaSuccess;
  if (grad_proj) {  // else ws.dldi already holds dL/dI * |X - s| (written by the step's forward)
    dim3 g((ws.nu * ws.nv + 255) / 256, ws.P);
    k_gpix<<<g, 256, 0, st>>>(grad_proj, views, ws.nu, ws.nv, ws.dldi);
    note_launches(1);
  }
  if (ws.bwd_lanes == 32) {
    const int units = (ws.n + kBwdThreads / 32 - 1) / (kBwdThreads / 32);
    dim3 grid((units + kBwdRounds - 1) / kBwdRounds, ws.P);
    k_raster_bwd<32><<<grid, kBwdThreads, 0, st>>>(ws.rec, ws.counts, ws.n, ws.nu, ws.nv, ws.dldi, c2, nullptr,
                                                   (float*)ws.grec, kBwdRounds);
  } else {
    const int G = (ws.n + 31) / 32;
    k_bwd_pairing<<<dim3((G + 7) / 8, ws.P), 256, 0, st>>>(ws.bcost, ws.counts, ws.n, G, ws.bperm);
    note_launches(1);
    const int units = (ws.n + kBwdThreads / 16 - 1) / (kBwdThreads / 16);
    dim3 grid((units + kBwdRounds - 1) / kBwdRounds, ws.P);
    k_raster_bwd<16><<<grid, kBwdThreads, 0, st>>>(ws.rec, ws.counts, ws.n, ws.nu, ws.nv, ws.dldi, c2, ws.bperm,
                                                   (float*)ws.grec, kBwdRounds);
  }
  note_launches(1);
  return cudaGetLastError();
}

// Sum of n partials in a fixed order: a block sums `chunk` consecutive values in one pass of its threads
// (strided), reduced by shuffles and through shared memory.  With more than one block, each block's sum
// replaces the first value of its own chunk (read only by that block) and one block then sums those.
__device__ __forceinline__ float block_sum_strided(const float* __restrict__ part, long long i0, long long i1,
                                                   long long stride) {
  __shared__ float red[32];
  float s = 0.f;
  for (long long i = i0 + (long long)threadIdx.x * stride; i < i1; i += (long long)blockDim.x * stride) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_loss_partial(float* __restrict__ part, long long n, long long chunk) {
  const long long i0 = (long long)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  const float t = block_sum_strided(part, i0, i1, 1);
  __syncthreads();  // every thread has read its values before the chunk's first one is replaced
  if (threadIdx.x == 0) part[i0] = t;
}

__global__ void __launch_bounds__(1024) k_loss_reduce(const float* __restrict__ part, long long n, long long stride,
                                                      float* out, float scale) {
  const float t = block_sum_strided(part, 0, n, stride);
  if (threadIdx.x == 0) out[0] = t * scale;
}

cudaError_t launch_loss_reduce(float* part, int n, float* out, float scale, cudaStream_t st) {
  // part holds per-warp sums of squared residuals; out[0] = scale * their sum (part is overwritten)
  constexpr long long kChunk = 2048;
  if (n <= 4 * kChunk) {
    k_loss_reduce<<<1, 1024, 0, st>>>(part, n, 1, out, scale);
    note_launches(1);
  } else {
    const long long blocks = (n + kChunk - 1) / kChunk;
    k_loss_partial<<<(unsigned)blocks, 256, 0, st>>>(part, n, kChunk);
    k_loss_reduce<<<1, 1024, 0, st>>>(part, n, kChunk, out, scale);
    note_launches(2);
  }
  return cudaGetLastError();
}

}  // namespace digs
