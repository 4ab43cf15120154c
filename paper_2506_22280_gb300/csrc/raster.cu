// Tile rasteriser of the X-ray transform (Sec. 3.1, Eq. 1, 3-4) and its backward pass.
//
// Work is done by half-warps (16 lanes), each sweeping one Gaussian's pixel box (or a 16-column slice
// of it) two pixels per lane per step in packed FP32x2 arithmetic (fma/mul/add.rn.f32x2).  Narrow
// slices (w <= 8): lane l owns column (l mod w), starts at row (l div w) and takes the row pair
// (r, r + s), s = 16 div w, stepping 2s rows.  Wider slices (8 < w <= 16): lane l owns the column pair
// (c, c + ceil(w/2)) of row (l div ceil(w/2)), stepping s = 16 div ceil(w/2) rows.  Per pixel, with
// (dx, dy) its offset from the projected mean:
//   num = dy (n11 dy + n01x2 dx) + n00 dx^2,  t = 1 + wn0 dx + wn1 dy,  D = t^2 + kappa num,  E = num / D.
// The only SFU operations per pixel are the exp2 and, unless D stays within 2 % of 1 over the box
// (then its binomial series through the cubic term is used in the forward), the reciprocal square root.
//
// Forward: one CTA per (projection, tile).  The tile's sorted Gaussian list is staged into shared
// memory in chunks of 256 records (48 B each) by 16-byte cp.async copies, double-buffered so the next
// chunk lands while the current one is processed; the thread that staged a record also derives, once,
// the part of the Gaussian's box inside the tile.  Each half-warp adds its Gaussians into its own tile
// canvas (no atomics); the 16 canvases merge in a fixed order, so the result is deterministic.
//
// Backward: needs no tile lists.  One half-warp per (projection, Gaussian) record sweeps the record's
// whole pixel box, reading g = dL/dI * |X - s| straight from the projection-sized image (L1/L2
// resident).  Each lane accumulates seven sums per pixel of its pair and turns them into the ten
// sufficient statistics of the record gradient; the half-warp reduces them with an 11-shuffle
// recursive halving and ten lanes write them to the record's slot (no atomics).
#include "digs_internal.h"

namespace digs {

constexpr int kRasterThreads = 256;
constexpr int kRasterWarps = kRasterThreads / 32;
constexpr int kChunk = kRasterThreads;
constexpr float kNegHalfLog2e = -0.5f * DIGS_LOG2E;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

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
// D^-1/2: binomial series (1 + e)^-1/2 ~ 1 - e/2 + 3e^2/8 - 5e^3/16 when |e| <= 0.02, else the SFU.
template <bool POLY>
__device__ __forceinline__ f2 f2_inv_sqrt(f2 D) {
  if (POLY) {
    f2 e = f2_add(D, f2_dup(-1.f));
    return f2_fma(e, f2_fma(e, f2_fma(e, f2_dup(-0.3125f), f2_dup(0.375f)), f2_dup(-0.5f)), f2_dup(1.f));
  }
  float a, b;
  f2_unpack(D, a, b);
  return f2_pack(sfu_rsqrt(a), sfu_rsqrt(b));
}

// ---- lane layouts (forward and backward) ---------------------------------------------------------

// Half-warp lane layout of a box slice w <= 16 pixels wide, per w: cw | s << 5 | m << 10, where cw is
// the number of lane columns, s the rows covered per pass and m = ceil(256 / cw), so that
// (l * m) >> 8 = l / cw exactly for l < 16.  w <= 8: lane l takes column l mod w and the row pair
// (r, r + s), s = 16 div w, stepping 2s rows.  8 < w <= 16: the column pair (c, c + ceil(w/2)),
// stepping s = 16 div ceil(w/2) rows.
struct HalfLaneTable {
  int v[17];
  constexpr HalfLaneTable() : v() {
    for (int w = 1; w <= 16; ++w) {
      const int cw = w <= 8 ? w : (w + 1) / 2;
      v[w] = cw | ((16 / cw) << 5) | (((256 + cw - 1) / cw) << 10);
    }
  }
};
__constant__ HalfLaneTable kHalfLanes = HalfLaneTable();

struct HalfLanes {
  int c, r0, pdx, pdy, ystep;
  bool active, col2;
};
__device__ __forceinline__ HalfLanes half_lanes(int w, int h, int hl) {
  const int t = kHalfLanes.v[w];
  const int cw = t & 31, s = (t >> 5) & 31, m = t >> 10;
  const int q = (hl * m) >> 8;
  const bool rows = w <= 8;
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

constexpr int kHalves = kRasterThreads / 16;  // half-warps per CTA, one canvas each

template <int TS>
struct RasterSmem {
  static constexpr size_t rec_bytes = 2 * kChunk * DIGS_REC_F4 * sizeof(float4);
  static constexpr size_t info_bytes = 2 * kChunk * sizeof(int4);
  static constexpr size_t head = rec_bytes + info_bytes;
  // Canvas rows are TS + 1 floats apart and consecutive canvases 16 banks apart, so the rows of one
  // half-warp's pixels and the two half-warps of a warp fall on different banks.
  static constexpr int pitch = TS + 1;
  static constexpr int canvas = TS * pitch + ((16 - (TS * pitch) % 32) + 32) % 32;
  static constexpr size_t fwd = head + kHalves * canvas * sizeof(float);
};

// Per-CTA staging state.
template <int TS>
struct Stage {
  float4* rec;    // [2][kChunk * 3] records
  int4* info;     // [2][kChunk]: (canvas offset y0 pitch + x0 | w << 11 | h << 17 | poly << 28, dx0, dy0, 0)
  __device__ void init(unsigned char* sm) {
    rec = (float4*)sm;
    info = (int4*)(sm + RasterSmem<TS>::rec_bytes);
  }
  // Enqueue the copies of chunk [base, end) into buffer `buf` (commits a group even when empty).
  __device__ void issue(const float4* __restrict__ grec, const uint32_t* __restrict__ srid, uint32_t base,
                        uint32_t end, int buf) {
    uint32_t k = base + threadIdx.x;
    if (k < end) {
      const float4* src = grec + (size_t)srid[k] * DIGS_REC_F4;
      float4* dst = rec + ((size_t)buf * kChunk + threadIdx.x) * DIGS_REC_F4;
#pragma unroll
      for (int q = 0; q < DIGS_REC_F4; ++q) cp_async16(dst + q, src + q);
    }
    cp_async_commit();
  }
  // After the chunk landed: this thread's record -> its box inside the tile.
  __device__ void derive(uint32_t base, uint32_t end, int buf, int ox, int oy) {
    uint32_t k = base + threadIdx.x;
    if (k >= end) return;
    const float4* r3 = rec + ((size_t)buf * kChunk + threadIdx.x) * DIGS_REC_F4;
    float4 a = r3[0], c = r3[2];
    int bx = __float_as_int(c.y), by = __float_as_int(c.z);
    int x0 = max(bx & 0xffff, ox) - ox, x1 = min(bx >> 16, ox + TS - 1) - ox;
    int y0 = max(by & 0xffff, oy) - oy, y1 = min(by >> 16, oy + TS - 1) - oy;
    int w = x1 - x0 + 1, h = y1 - y0 + 1;
    if (w <= 0 || h <= 0) { w = 1; h = 0; x0 = 0; y0 = 0; }  // keys come from the box: kept as a guard
    int packed = (y0 * RasterSmem<TS>::pitch + x0) | (w << 11) | (h << 17) | ((__float_as_int(c.w) & 1) << 28);
    info[buf * kChunk + threadIdx.x] = make_int4(packed, __float_as_int((float)(ox + x0) - a.x),
                                                 __float_as_int((float)(oy + y0) - a.y), 0);
  }
};

// Forward over the lane's pixel pairs of one box slice; p points at the lane's first pixel in the
// half-warp's canvas.
template <int TS, bool POLY, bool COUNT>
__device__ __forceinline__ void fwd_pixels(const float4* r3, const HalfLanes& B, int h, float dx1, float dy1,
                                           float* p, float c2, unsigned& n_cut) {
  const float4 ra = r3[0], rb = r3[1];
  const float amp = r3[2].x;
  const float dx2 = dx1 + (float)B.pdx;
  const f2 DX = f2_pack(dx1, dx2);
  const f2 A = f2_mul(f2_mul(f2_dup(ra.z), DX), DX), BQ = f2_mul(f2_dup(ra.w), DX);
  const f2 T0 = f2_fma(f2_dup(rb.y), DX, f2_dup(1.f));
  const f2 N11 = f2_dup(rb.x), WN1 = f2_dup(rb.z), KAP = f2_dup(rb.w), AMP = f2_dup(amp);
  const f2 C2 = f2_dup(c2), KNEG = f2_dup(kNegHalfLog2e), STEP = f2_dup((float)B.ystep);
  constexpr int pitch = RasterSmem<TS>::pitch;
  const int pstep = B.ystep * pitch, d2 = B.pdy * pitch + B.pdx, hb = B.col2 ? h - B.pdy : 0;
  f2 DY = f2_pack(dy1, dy1 + (float)B.pdy);
  for (int r = B.r0; r < h; r += B.ystep, DY = f2_add(DY, STEP), p += pstep) {
    f2 NUM = f2_fma(DY, f2_fma(N11, DY, BQ), A);
    f2 T = f2_fma(WN1, DY, T0);
    f2 D = f2_fma(T, T, f2_mul(KAP, NUM));
    f2 RS = f2_inv_sqrt<POLY>(D);
    f2 EX = f2_exp2(f2_mul(f2_mul(NUM, f2_mul(RS, RS)), KNEG));
    f2 VAL = f2_mul(f2_mul(AMP, RS), EX);
    f2 LIM = f2_mul(C2, D);
    float na, nb, la, lb, va, vb;
    f2_unpack(NUM, na, nb);
    f2_unpack(LIM, la, lb);
    f2_unpack(VAL, va, vb);
    if (na <= la) {  // E = num / D <= cutoff^2
      p[0] += va;
      if (COUNT) ++n_cut;
    }
    if (r < hb && nb <= lb) {  // the partner lies inside the box part in this tile
      p[d2] += vb;
      if (COUNT) ++n_cut;
    }
  }
}

// One CTA per (projection, tile); each half-warp takes one staged entry at a time and adds it into its
// own canvas; the 16 canvases are merged in a fixed order.
template <int TS, bool COUNT>
__global__ void __launch_bounds__(kRasterThreads) k_raster_fwd(
    const float4* __restrict__ grec, const uint32_t* __restrict__ srid, const uint2* __restrict__ ranges,
    const __grid_constant__ ViewsParam views, int tiles_x, int T, int nu, int nv, float c2, float* __restrict__ proj,
    const float* __restrict__ meas, float* __restrict__ dldi, float* __restrict__ loss_part, float inv_count,
    unsigned long long* __restrict__ counters) {
  extern __shared__ __align__(16) unsigned char smem[];
  Stage<TS> S;
  S.init(smem);
  constexpr int pitch = RasterSmem<TS>::pitch, canvas = RasterSmem<TS>::canvas;
  float* acc = (float*)(smem + RasterSmem<TS>::head);  // [kHalves][canvas]
  __shared__ float red[kRasterWarps];
  const int b = blockIdx.y, tile = blockIdx.x;
  const int ox = (tile % tiles_x) * TS, oy = (tile / tiles_x) * TS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, hl = threadIdx.x & 15;
  for (int p = threadIdx.x; p < kHalves * canvas; p += kRasterThreads) acc[p] = 0.f;
  const uint2 rg = ranges[(size_t)b * T + tile];
  const ViewC& v = views.v[b];
  float* acch = acc + (threadIdx.x >> 4) * canvas;
  unsigned n_box = 0, n_cut = 0;
  if (rg.x < rg.y) S.issue(grec, srid, rg.x, rg.y, 0);
  for (uint32_t base = rg.x, it = 0; base < rg.y; base += kChunk, ++it) {
    const int buf = it & 1;
    S.issue(grec, srid, base + kChunk, rg.y, buf ^ 1);
    cp_async_wait_prev();
    S.derive(base, rg.y, buf, ox, oy);
    __syncthreads();
    const int cnt = min((int)(rg.y - base), kChunk);
    for (int e0 = 2 * warp; e0 < cnt; e0 += kHalves) {  // warp-uniform trip count
      const int e = e0 + ((threadIdx.x >> 4) & 1);
      const bool has = e < cnt;
      const int4 inf = S.info[buf * kChunk + (has ? e : e0)];
      const int w = has ? (inf.x >> 11) & 63 : 0, h = (inf.x >> 17) & 63;
      const bool poly = __all_sync(0xffffffffu, !has || ((inf.x >> 28) & 1));
      if (COUNT && hl == 0) n_box += w * h;
      const float4* r3 = S.rec + ((size_t)buf * kChunk + e) * DIGS_REC_F4;
      for (int cx = 0; cx < w; cx += 16) {  // 16-column slices (one unless TS = 32)
        const HalfLanes B = half_lanes(min(16, w - cx), h, hl);
        if (B.active) {
          const float dx1 = __int_as_float(inf.y) + (float)(cx + B.c), dy1 = __int_as_float(inf.z) + (float)B.r0;
          float* p = acch + (inf.x & 2047) + B.r0 * pitch + cx + B.c;
          if (poly)
            fwd_pixels<TS, true, COUNT>(r3, B, h, dx1, dy1, p, c2, n_cut);
          else
            fwd_pixels<TS, false, COUNT>(r3, B, h, dx1, dy1, p, c2, n_cut);
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  float lsum = 0.f;
  for (int p = threadIdx.x; p < TS * TS; p += kRasterThreads) {
    int px = ox + p % TS, py = oy + p / TS;
    if (px < nu && py < nv) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < kHalves; ++q) s += acc[q * canvas + (p / TS) * pitch + p % TS];
      const float lp = pixel_ray_length(v, (float)px, (float)py);
      float I = s * lp;
      size_t idx = ((size_t)b * nv + py) * nu + px;
      if (proj) proj[idx] = I;
      if (meas) {
        float res = I - meas[idx];
        lsum = fmaf(res, res, lsum);
        if (dldi) dldi[idx] = 2.f * res * inv_count * lp;  // dL/dI * |X - s|, what the backward consumes
      }
    }
  }
  if (COUNT) {
    unsigned c = n_cut;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    n_box += __shfl_xor_sync(0xffffffffu, n_box, 16);  // lanes 0 and 16 counted their half-warp's boxes
    if (lane == 0 && (n_box | c)) {
      atomicAdd(counters, (unsigned long long)n_box);
      atomicAdd(counters + 1, (unsigned long long)c);
    }
  }
  if (loss_part) {
    lsum = warp_sum(lsum);
    if (lane == 0) red[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int q = 0; q < kRasterWarps; ++q) s += red[q];
      loss_part[(size_t)b * T + tile] = s;
    }
  }
}

// ---- backward: one half-warp per (projection, Gaussian) record, over the record's whole pixel box ----

constexpr int kBwdThreads = 256;
constexpr int kBwdRecords = kBwdThreads / 16;  // records per CTA

// Adds the lane's share of the ten record-gradient sums, all but the first divided by amp / 2:
// sum g V/amp; sum dL/dnum (dx^2, dx dy, dy^2); sum dL/dnum (dx, dy); sum dL/dt (1, dx, dy);
// sum dL/dkappa.  gp points at g = dL/dI * |X - s| of the lane's first pixel in the projection image
// (row pitch nu); (dx1, dy1) is that pixel's offset from the projected mean.
__device__ __forceinline__ void bwd_box_pixels(const Rec& R0, const HalfLanes& B, int h, float dx1, float dy1,
                                               const float* __restrict__ gp, int nu, float c2, float Sv[10]) {
  const float dx2 = dx1 + (float)B.pdx;
  const f2 DX = f2_pack(dx1, dx2);
  const f2 AQ = f2_mul(f2_mul(f2_dup(R0.n00), DX), DX), BQ = f2_mul(f2_dup(R0.n01x2), DX);
  const f2 T0 = f2_fma(f2_dup(R0.wn0), DX, f2_dup(1.f));
  const f2 N11 = f2_dup(R0.n11), WN1 = f2_dup(R0.wn1), KAP = f2_dup(R0.kappa);
  const f2 KNEG = f2_dup(kNegHalfLog2e), MONE = f2_dup(-1.f), STEP = f2_dup((float)B.ystep);
  const int pstep = B.ystep * nu, d2 = B.pdy * nu + B.pdx;
  f2 DY = f2_pack(dy1, dy1 + (float)B.pdy);
  f2 S0 = f2_dup(0.f), S1 = S0, S2 = S0, S3 = S0, S4 = S0, S5 = S0, S6 = S0;
  for (int r = B.r0; r < h; r += B.ystep, DY = f2_add(DY, STEP), gp += pstep) {
    f2 NUM = f2_fma(DY, f2_fma(N11, DY, BQ), AQ);
    f2 T = f2_fma(WN1, DY, T0);
    f2 D = f2_fma(T, T, f2_mul(KAP, NUM));
    f2 RS = f2_inv_sqrt<false>(D);
    f2 INVD = f2_mul(RS, RS);
    f2 E = f2_mul(NUM, INVD);
    f2 BV = f2_mul(RS, f2_exp2(f2_mul(E, KNEG)));      // V / amp
    float na, nb, da, db;
    f2_unpack(NUM, na, nb);
    f2_unpack(D, da, db);
    const float ga = (na <= c2 * da) ? __ldg(gp) : 0.f;                                     // E <= cutoff^2
    const float gb = (B.col2 && r + B.pdy < h && nb <= c2 * db) ? __ldg(gp + d2) : 0.f;  // partner in the box
    f2 G = f2_pack(ga, gb);
    S0 = f2_fma(G, BV, S0);
    f2 AL = f2_mul(G, f2_mul(BV, INVD));                     // (dL/dV * V / (2 D)) / (amp / 2)
    f2 EM1 = f2_add(E, MONE);
    f2 GNUM = f2_mul(AL, f2_fma(KAP, EM1, MONE));          // dL/dnum
    f2 AEM = f2_mul(AL, EM1);
    f2 GTH = f2_mul(AEM, T);                                 // (dL/dt) / 2
    f2 GND = f2_mul(GNUM, DY);
    S1 = f2_add(S1, GNUM);
    S2 = f2_add(S2, GND);
    S3 = f2_fma(GND, DY, S3);
    S4 = f2_add(S4, GTH);
    S5 = f2_fma(GTH, DY, S5);
    S6 = f2_fma(AEM, NUM, S6);                               // dL/dkappa
  }
  // each pixel of the pair keeps its column, so its dx-moments follow from its dy-moments
  float a[7][2];
  const f2 Sp[7] = {S0, S1, S2, S3, S4, S5, S6};
#pragma unroll
  for (int i = 0; i < 7; ++i) f2_unpack(Sp[i], a[i][0], a[i][1]);
  const float dxs[2] = {dx1, dx2};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float dx = dxs[j];
    Sv[0] += a[0][j];
    Sv[1] += dx * dx * a[1][j];
    Sv[2] += dx * a[2][j];
    Sv[3] += a[3][j];
    Sv[4] += dx * a[1][j];
    Sv[5] += a[2][j];
    Sv[6] += 2.f * a[4][j];
    Sv[7] += 2.f * dx * a[4][j];
    Sv[8] += 2.f * a[5][j];
    Sv[9] += a[6][j];
  }
}

// Sum ten per-lane values over each half-warp (lanes hl = 0..15) and store them to out[0..9].
// Recursive halving over an uneven split, 5 + 3 + 2 + 1 shuffles: after the xor-8 exchange a lane
// holds five values (0-4 or 5-9), after xor-4 three of those five (local 0-2, or 3-4 plus a pad),
// after xor-2 two, after xor-1 one, the value 5 b3 + 3 b2 + 2 b1 + b0 (b_k = bit k of hl) when that
// lies inside its group of five.
__device__ __forceinline__ void half_reduce_store10(const float v[10], float* out, int hl, bool store) {
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
  const float d = (hi ? c1 : c0) + __shfl_xor_sync(full, hi ? c0 : c1, 1);
  const int bit2 = (hl >> 2) & 1;
  const int local = 3 * bit2 + 2 * ((hl >> 1) & 1) + (hl & 1);
  if (store && local < (bit2 ? 5 : 3)) out[((hl & 8) ? 5 : 0) + local] = d;
}

// One half-warp per (projection, Gaussian) record: the ten sums over every pixel of the record's box,
// reduced over the half-warp and written to grec[record] (12 floats, the last two unused).  Records
// whose Gaussian was culled get zeros.  Grid: (ceil(N / 16), P).
__global__ void __launch_bounds__(kBwdThreads, 4) k_raster_bwd(const float4* __restrict__ rec,
                                                                const uint32_t* __restrict__ counts, int N, int nu,
                                                                int nv, const float* __restrict__ gpix, float c2,
                                                                float* __restrict__ grec) {
  const int hl = threadIdx.x & 15;
  const int b = blockIdx.y;
  const int n = blockIdx.x * kBwdRecords + (threadIdx.x >> 4);
  const bool valid = n < N;
  const size_t i = (size_t)b * N + (valid ? n : 0);
  float Sv[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (valid && counts[i] != 0u) {
    const Rec R0 = load_rec(rec + i * DIGS_REC_F4);
    const int x0 = R0.bx & 0xffff, x1 = R0.bx >> 16, y0 = R0.by & 0xffff, y1 = R0.by >> 16;
    const int w = x1 - x0 + 1, h = y1 - y0 + 1;
    const float* gimg = gpix + (size_t)b * nv * nu;
    for (int cx = 0; cx < w; cx += 16) {  // boxes wider than 16 pixels: 16-column slices
      const HalfLanes B = half_lanes(min(16, w - cx), h, hl);
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
  half_reduce_store10(Sv, grec + i * (DIGS_PARTIAL_F4 * 4), hl, valid);
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
  const size_t smem = RasterSmem<TS>::fwd;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_raster_fwd<TS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_raster_fwd<TS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  dim3 grid(ws.T, ws.P);
  float* lp = meas ? ws.loss_part : nullptr;
  if (count)
    k_raster_fwd<TS, true><<<grid, kRasterThreads, smem, st>>>(ws.rec, ws.srid, ws.ranges, views, ws.tiles_x, ws.T,
                                                                ws.nu, ws.nv, c2, proj, meas, dldi, lp, inv_count,
                                                                ws.counters);
  else
    k_raster_fwd<TS, false><<<grid, kRasterThreads, smem, st>>>(ws.rec, ws.srid, ws.ranges, views, ws.tiles_x, ws.T,
                                                                 ws.nu, ws.nv, c2, proj, meas, dldi, lp, inv_count,
                                                                 ws.counters);
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
  dim3 grid((ws.n + kBwdRecords - 1) / kBwdRecords, ws.P);
  k_raster_bwd<<<grid, kBwdThreads, 0, st>>>(ws.rec, ws.counts, ws.n, ws.nu, ws.nv, ws.dldi, c2, (float*)ws.grec);
  note_launches(1);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_loss_reduce(const float* __restrict__ part, int n, float* out,
                                                      float scale) {
  __shared__ float red[32];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[0] = t * scale;
  }
}

cudaError_t launch_loss_reduce(const float* part, int n, float* out, float scale, cudaStream_t st) {
  // part holds per-tile sums of squared residuals; out[0] = scale * their sum
  k_loss_reduce<<<1, 1024, 0, st>>>(part, n, out, scale);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace digs
