// C-ABI entry points of libdigs: argument checks, workspace carve-up, per-view constants (derived in
// double precision on the host) and the launch sequences of the forward / backward passes and the step.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "digs_internal.h"

#include <atomic>

namespace digs {

static std::atomic<long long> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t layout(Workspace* ws, void* base, int n, int P, int nu, int nv, int R, long long cap, int tile,
              int n_total, int w_rows) {
  Workspace w;
  memset(&w, 0, sizeof(w));
  w.n = n; w.n_total = n_total; w.P = P; w.nu = nu; w.nv = nv; w.R = R; w.cap = cap; w.tile = tile;
  w.tiles_x = (nu + tile - 1) / tile;
  w.tiles_y = (nv + tile - 1) / tile;
  w.T = w.tiles_x * w.tiles_y;
  w.n_sort_blocks = sort_blocks(cap, P);
  size_t PN = (size_t)P * n;
  size_t off = 0;
  char* b = (char*)base;
  auto take = [&](size_t bytes) -> char* {
    char* p = b ? b + off : nullptr;
    off += align256(bytes);
    return p;
  };
  w.status = (int*)take(256);
  w.n_pairs = (uint32_t*)(w.status ? (char*)w.status + 64 : nullptr);
  w.counters = (unsigned long long*)(w.status ? (char*)w.status + 128 : nullptr);
  w.rec = (float4*)take(PN * DIGS_REC_F4 * sizeof(float4));
  w.counts = (uint32_t*)take((PN + 1) * 4);
  w.n_chunks = bin_chunks(n, w.T);
  if (w.n_chunks > 0 && (size_t)P * w.T * w.n_chunks >= ((size_t)1 << 30)) w.n_chunks = -1;  // scan length is an int
  const size_t chist_n = (size_t)P * w.T * std::max(w.n_chunks, 0);
  w.tbox = (uint2*)take(PN * sizeof(uint2));
  w.chist = (uint32_t*)take((chist_n + 1) * 4);
  w.offsets = (uint32_t*)take((PN + 1) * 4);
  size_t tmp = std::max(scan_tmp_words((int)PN), scan_tmp_words(256 * std::max(w.n_sort_blocks, 1)));
  tmp = std::max(tmp, scan_tmp_words((int)chist_n));
  w.scan_tmp = (uint32_t*)take(tmp * 4);
  w.keys = (uint32_t*)take((size_t)cap * 4);
  w.vals = (uint32_t*)take((size_t)cap * 4);
  w.keys_alt = (uint32_t*)take((size_t)cap * 4);
  w.vals_alt = (uint32_t*)take((size_t)cap * 4);
  w.hist = (uint32_t*)take(((size_t)256 * w.n_sort_blocks + 1) * 4);
  w.seg = (uint32_t*)take(((size_t)2 * P + 2) * 4);
  w.ranges = (uint2*)take((size_t)P * w.T * sizeof(uint2));
  w.order = (uint32_t*)take((size_t)P * w.T * 4);
  w.grec = (float4*)take(PN * DIGS_PARTIAL_F4 * sizeof(float4));
  w.bcost = (uint8_t*)take(PN);
  w.bperm = (uint8_t*)take((size_t)P * ((n + 31) / 32) * 32);
  w.gw_part = (float*)take((size_t)pair_sum_blocks(n_total) * P * R * 4 + 4);
  w.loss_part = (float*)take((size_t)P * w.T * fwd_blocks(tile) * 4 + 4);
  w.ffd = (float*)take((size_t)12 * R * n_total * 4 + 4);
  w.ffd2 = (float*)take((size_t)18 * R * n_total * 4 + 4);
  w.gsum = (float*)take((size_t)(11 + 12 * R) * n_total * 4 + 4);
  w.proj = (float*)take((size_t)P * nu * nv * 4);
  w.dldi = (float*)take((size_t)P * nu * nv * 4);
  w.gw_rows = (float*)take((size_t)w_rows * R * 4 + 4);
  w.bytes = off;
  if (ws) *ws = w;
  return off;
}

}  // namespace digs

using namespace digs;

namespace {

#define DIGS_TRY(expr)                        \
  do {                                        \
    cudaError_t e__ = (expr);                 \
    if (e__ != cudaSuccess) return DIGS_ERR_CUDA; \
  } while (0)

int opt_tile(const DigsOpts* o) { return (o && o->tile) ? o->tile : 16; }
float opt_c2(const DigsOpts* o) {
  float c = (o && o->cutoff > 0.f) ? o->cutoff : 3.5f;
  return c * c;
}
bool opt_valid(const DigsOpts* o) {
  if (!o) return true;
  if (!(o->cutoff >= 0.f) || !isfinite(o->cutoff)) return false;
  int t = o->tile, l = o->bwd_lanes;
  return (t == 0 || t == 8 || t == 16 || t == 32) && (l == 0 || l == 16 || l == 32);
}

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

digs_status make_view(const DigsView& in, int w_row, ViewC& v) {
  const double* arrs[4] = {in.src, in.det_c, in.e_u, in.e_v};
  for (auto a : arrs)
    for (int i = 0; i < 3; ++i)
      if (!isfinite(a[i])) return DIGS_ERR_ARG;
  if (!(in.du > 0) || !(in.dv > 0) || !isfinite(in.off_u) || !isfinite(in.off_v)) return DIGS_ERR_ARG;
  if (in.nu < 1 || in.nv < 1 || in.nu > 32767 || in.nv > 32767) return DIGS_ERR_ARG;
  if (fabs(dot3(in.e_u, in.e_u) - 1) > 1e-6 || fabs(dot3(in.e_v, in.e_v) - 1) > 1e-6 ||
      fabs(dot3(in.e_u, in.e_v)) > 1e-6)
    return DIGS_ERR_ARG;
  double n[3] = {in.e_u[1] * in.e_v[2] - in.e_u[2] * in.e_v[1], in.e_u[2] * in.e_v[0] - in.e_u[0] * in.e_v[2],
                 in.e_u[0] * in.e_v[1] - in.e_u[1] * in.e_v[0]};
  double sd[3] = {in.det_c[0] - in.src[0], in.det_c[1] - in.src[1], in.det_c[2] - in.src[2]};
  double sdd = sqrt(dot3(sd, sd));
  if (!(sdd > 0)) return DIGS_ERR_ARG;
  if (dot3(n, sd) < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
  const double* fr[3] = {in.e_u, in.e_v, n};
  double dir[3] = {sd[0] / sdd, sd[1] / sdd, sd[2] / sdd};
  for (int c = 0; c < 3; ++c) {
    for (int k = 0; k < 3; ++k) v.F[3 * c + k] = (float)fr[c][k];
    v.src_d[c] = (float)dot3(fr[c], in.src);
    v.det_d[c] = (float)dot3(fr[c], in.det_c);
    v.dir_d[c] = (float)dot3(fr[c], dir);
  }
  v.su = (float)(-dot3(in.e_u, sd));
  v.sv = (float)(-dot3(in.e_v, sd));
  v.sdd_n = (float)dot3(n, sd);
  if (!(v.sdd_n > 0.f)) return DIGS_ERR_ARG;
  v.du = (float)in.du; v.dv = (float)in.dv;
  v.inv_du = (float)(1.0 / in.du); v.inv_dv = (float)(1.0 / in.dv);
  v.cx0 = (float)((in.nu - 1) * 0.5 - in.off_u);
  v.cy0 = (float)((in.nv - 1) * 0.5 - in.off_v);
  v.nu = in.nu; v.nv = in.nv;
  v.parallel = in.parallel ? 1 : 0;
  if (v.parallel && !(v.dir_d[2] > 0.f)) return DIGS_ERR_ARG;
  v.w_row = w_row;
  return DIGS_OK;
}

digs_status make_lattice(const DigsLattice* lat, LatticeC& L) {
  if (!lat || lat->R < 1 || lat->R > DIGS_MAX_R || lat->nx < 1 || lat->ny < 1 || lat->nz < 1) return DIGS_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (!(lat->spacing[a] > 0.f) || !isfinite(lat->spacing[a]) || !isfinite(lat->origin[a])) return DIGS_ERR_ARG;
    L.origin[a] = lat->origin[a];
    L.inv_h[a] = 1.f / lat->spacing[a];
  }
  L.nx = lat->nx; L.ny = lat->ny; L.nz = lat->nz; L.R = lat->R;
  return DIGS_OK;
}

// Largest pair capacity whose layout fits `bytes` (n: record stride, n_total: all Gaussians).
long long capacity_for(size_t bytes, int n, int P, int nu, int nv, int R, int tile, int n_total, int w_rows) {
  if (layout(nullptr, nullptr, n, P, nu, nv, R, 0, tile, n_total, w_rows) > bytes) return -1;
  long long lo = 0, hi = 1;
  while (layout(nullptr, nullptr, n, P, nu, nv, R, hi, tile, n_total, w_rows) <= bytes && hi < (1LL << 32)) hi *= 2;
  while (hi - lo > 1) {
    long long mid = (lo + hi) / 2;
    if (layout(nullptr, nullptr, n, P, nu, nv, R, mid, tile, n_total, w_rows) <= bytes) lo = mid; else hi = mid;
  }
  return std::min(lo, (long long)0xffffffffLL);
}

size_t phi_floats(const LatticeC& L) { return (size_t)L.nx * L.ny * L.nz * 3 * L.R; }

ScanTable one_scan(int n, const LatticeC& L) {
  ScanTable t;
  memset(&t, 0, sizeof(t));
  t.S = 1;
  t.off[1] = n;
  for (int k = 2; k <= DIGS_MAX_SCANS; ++k) t.off[k] = n;
  t.nmax = n;
  t.phi_stride = (long long)phi_floats(L);
  return t;
}

// The scans of a state: n_scans <= 1 is one scan of all n Gaussians.
digs_status state_scans(const DigsState* st, const LatticeC& L, ScanTable& t) {
  t = one_scan(st->n, L);
  if (st->n_scans <= 1) return DIGS_OK;
  if (st->n_scans > DIGS_MAX_SCANS) return DIGS_ERR_ARG;
  if (st->scan_off[0] != 0 || st->scan_off[st->n_scans] != st->n) return DIGS_ERR_ARG;
  t.S = st->n_scans;
  t.nmax = 0;
  for (int s = 0; s < t.S; ++s) {
    if (st->scan_off[s + 1] < st->scan_off[s]) return DIGS_ERR_ARG;
    t.off[s] = st->scan_off[s];
    t.nmax = std::max(t.nmax, st->scan_off[s + 1] - st->scan_off[s]);
  }
  for (int k = t.S; k <= DIGS_MAX_SCANS; ++k) t.off[k] = st->n;
  return DIGS_OK;
}

struct Call {
  GaussPtrs g;
  ScanTable sc;
  LatticeC L;
  ViewsParam views;
  Workspace ws;
  float c2;
  int P;
  int flags;
  cudaStream_t st;
};

// Stage events of the most recent call made with DIGS_FLAG_TIME_STAGES (process-wide, diagnostic).
cudaEvent_t g_ev[DIGS_NUM_STAGES + 1];
bool g_ev_ready = false;
unsigned g_ev_marked = 0;

// Record the boundary `i` (stage i - 1 ends, stage i starts) when the call is timed.
void mark(const Call& c, int i) {
  if (!(c.flags & DIGS_FLAG_TIME_STAGES)) return;
  if (!g_ev_ready) {
    for (auto& e : g_ev) cudaEventCreate(&e);
    g_ev_ready = true;
  }
  if (i == 0) g_ev_marked = 0;
  cudaEventRecord(g_ev[i], c.st);
  g_ev_marked |= 1u << i;
}

// scans: the state's scan table (digs_step), else nullptr for one scan of all g->n Gaussians.
digs_status prepare(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                    const DigsView* views, int P, const DigsOpts* opts, const int* rows, void* wsp, size_t ws_bytes,
                    void* stream, Call& c, const DigsState* scans = nullptr) {
  if (!g || !views || P < 0 || P > DIGS_MAX_VIEWS || g->n < 0 || !opt_valid(opts)) return DIGS_ERR_ARG;
  if (g->n > 0 && (!g->mu0 || !g->scale || !g->quat || !g->rho)) return DIGS_ERR_ARG;
  if (!phi || !w || !wsp) return DIGS_ERR_ARG;
  if (((uintptr_t)wsp & 255) != 0) return DIGS_ERR_ARG;
  digs_status s = make_lattice(lat, c.L);
  if (s != DIGS_OK) return s;
  if (scans) {
    s = state_scans(scans, c.L, c.sc);
    if (s != DIGS_OK) return s;
  } else {
    c.sc = one_scan(g->n, c.L);
  }
  int nu = P > 0 ? views[0].nu : 1, nv = P > 0 ? views[0].nv : 1;
  for (int b = 0; b < P; ++b) {
    if (views[b].nu != nu || views[b].nv != nv) return DIGS_ERR_ARG;
    s = make_view(views[b], rows ? rows[b] : b, c.views.v[b]);
    if (s != DIGS_OK) return s;
    c.views.v[b].ewa = (opts && (opts->flags & DIGS_FLAG_EWA) && !views[b].parallel) ? 1 : 0;
    const int sc = scans ? views[b].scan : 0;
    if (sc < 0 || sc >= c.sc.S) return DIGS_ERR_ARG;
    c.views.v[b].scan = sc;
  }
  c.g = GaussPtrs{g->mu0, g->scale, g->quat, g->rho, g->n};
  c.c2 = opt_c2(opts);
  c.P = P;
  c.flags = opts ? opts->flags : 0;
  c.st = (cudaStream_t)stream;
  int tile = opt_tile(opts);
  const int w_rows = (scans && scans->w_ctrl) ? scans->n_w : 0;
  long long cap = capacity_for(ws_bytes, c.sc.nmax, P, nu, nv, c.L.R, tile, g->n, w_rows);
  if (cap < 0) return DIGS_ERR_ARG;
  layout(&c.ws, wsp, c.sc.nmax, P, nu, nv, c.L.R, cap, tile, g->n, w_rows);
  c.ws.bwd_lanes = (opts && opts->bwd_lanes == 32) ? 32 : 16;
  return DIGS_OK;
}

// Warp, projection set-up and the per-pair records (all the backward needs).
digs_status prep(Call& c, const float* phi, const float* w) {
  Workspace& ws = c.ws;
  mark(c, 0);
  DIGS_TRY(cudaMemsetAsync(ws.counters, 0, 2 * sizeof(unsigned long long), c.st));
  DIGS_TRY(launch_prep_fwd(c.g, c.sc, c.L, phi, w, c.views, c.P, c.c2, ws, c.st));
  mark(c, 1);
  return DIGS_OK;
}

// Steps up to the sorted tile lists (what the forward raster needs).
digs_status bin(Call& c, const float* phi, const float* w) {
  Workspace& ws = c.ws;
  digs_status s = prep(c, phi, w);
  if (s != DIGS_OK) return s;
  if (ws.n_chunks >= 0) {  // counting sort straight from the records (T <= kDirectMaxTiles)
    DIGS_TRY(bin_direct(ws, c.st));
    ws.srid = ws.vals;
    mark(c, 2);
  } else {  // emitted (key, record) pairs and a radix sort of the tile index
    DIGS_TRY(exclusive_scan(ws.counts, ws.offsets, c.P * ws.n, ws.scan_tmp, c.st));
    DIGS_TRY(launch_emit(ws, c.st));
    mark(c, 2);
    uint32_t *sk = nullptr, *sv = nullptr;
    DIGS_TRY(sort_pairs(ws.keys, ws.vals, ws.keys_alt, ws.vals_alt, ws.n_pairs, ws.cap, ws.offsets, ws.n, c.P,
                        ws.T, ws.n_sort_blocks, ws.seg, ws.hist, ws.scan_tmp, ws.ranges, &sk, &sv, c.st));
    ws.srid = sv;
  }
  DIGS_TRY(tile_order(ws.ranges, c.P * ws.T, ws.order, c.st));
  mark(c, 3);
  return DIGS_OK;
}

// grad_proj = dL/dI, or nullptr when ws.dldi already holds dL/dI * |X - s|.
digs_status backward(Call& c, const float* phi, const float* w, const float* grad_proj, float* g_mu0,
                     float* g_scale, float* g_quat, float* g_rho, float* g_phi, float* g_w, int w_rows,
                     float* dens_grad = nullptr) {
  DIGS_TRY(cudaMemsetAsync(g_phi, 0, c.sc.S * phi_floats(c.L) * sizeof(float), c.st));
  mark(c, 5);
  if (c.g.n > 0) DIGS_TRY(launch_raster_bwd(c.ws, c.views, c.c2, grad_proj, c.st));
  mark(c, 6);
  if (c.g.n > 0)
    DIGS_TRY(launch_chain_bwd(c.g, c.sc, c.L, phi, w, c.views, c.P, c.ws, g_mu0, g_scale, g_quat, g_rho, g_phi,
                              dens_grad, c.st));
  DIGS_TRY(launch_gw_reduce(c.ws, c.views, c.P, c.L.R, g_w, w_rows, c.st));
  mark(c, 7);
  return DIGS_OK;
}

}  // namespace

extern "C" {

size_t digs_workspace_size(int n, int P, int nu, int nv, int R, long long max_pairs, const DigsOpts* opts) {
  if (n < 0 || P < 0 || nu < 1 || nv < 1 || R < 1 || R > DIGS_MAX_R || max_pairs < 0 || !opt_valid(opts)) return 0;
  return layout(nullptr, nullptr, n, P, nu, nv, R, max_pairs, opt_tile(opts), n);
}

size_t digs_state_workspace_size(const DigsState* st, int B, int nu, int nv, long long max_pairs,
                                 const DigsOpts* opts) {
  if (!st || B < 0 || nu < 1 || nv < 1 || max_pairs < 0 || !opt_valid(opts)) return 0;
  LatticeC L;
  ScanTable t;
  if (make_lattice(&st->lat, L) != DIGS_OK || state_scans(st, L, t) != DIGS_OK) return 0;
  return layout(nullptr, nullptr, t.nmax, B, nu, nv, L.R, max_pairs, opt_tile(opts), st->n,
                st->w_ctrl ? st->n_w : 0);
}

size_t digs_state_size(const DigsState* st) {
  if (!st) return 0;
  const size_t wg = st->w_ctrl ? (size_t)st->n_ctrl * st->lat.R : (size_t)st->n_w * st->lat.R;
  const size_t S = st->n_scans > 1 ? (size_t)st->n_scans : 1;
  return (size_t)st->n * 11 + S * st->lat.nx * st->lat.ny * st->lat.nz * 3 * st->lat.R + wg;
}

digs_status digs_ffd_eval(const DigsLattice* lat, const float* phi, const float* x, int n, float* U, float* dU,
                          void* stream) {
  LatticeC L;
  digs_status s = make_lattice(lat, L);
  if (s != DIGS_OK) return s;
  if (n < 0 || (n > 0 && (!phi || !x || !U || !dU))) return DIGS_ERR_ARG;
  DIGS_TRY(launch_ffd_eval(L, phi, x, n, U, dU, (cudaStream_t)stream));
  return DIGS_OK;
}

digs_status digs_count_pairs(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                             const DigsView* views, int P, const DigsOpts* opts, void* ws, size_t ws_bytes,
                             long long* count_host, void* stream) {
  if (!count_host) return DIGS_ERR_ARG;
  Call c;
  digs_status s = prepare(g, lat, phi, w, views, P, opts, nullptr, ws, ws_bytes, stream, c);
  if (s != DIGS_OK) return s;
  DIGS_TRY(launch_prep_fwd(c.g, c.sc, c.L, phi, w, c.views, c.P, c.c2, c.ws, c.st));
  DIGS_TRY(exclusive_scan(c.ws.counts, c.ws.offsets, c.P * c.ws.n, c.ws.scan_tmp, c.st));
  uint32_t total = 0;
  DIGS_TRY(cudaMemcpyAsync(&total, c.ws.offsets + (size_t)c.P * c.ws.n, 4, cudaMemcpyDeviceToHost, c.st));
  DIGS_TRY(cudaStreamSynchronize(c.st));
  *count_host = (long long)total;
  return DIGS_OK;
}

digs_status digs_project_fwd(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                             const DigsView* views, int P, const DigsOpts* opts, float* proj, void* ws,
                             size_t ws_bytes, void* stream) {
  Call c;
  digs_status s = prepare(g, lat, phi, w, views, P, opts, nullptr, ws, ws_bytes, stream, c);
  if (s != DIGS_OK) return s;
  if (P == 0) return DIGS_OK;
  if (!proj) return DIGS_ERR_ARG;
  s = bin(c, phi, w);
  if (s != DIGS_OK) return s;
  DIGS_TRY(launch_raster_fwd(c.ws, c.views, c.c2, proj, nullptr, nullptr, 0.f, c.st));
  mark(c, 4);
  return DIGS_OK;
}

digs_status digs_project_loss(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                              const DigsView* views, int P, const DigsOpts* opts, const float* meas, float* proj,
                              float* loss_out, void* ws, size_t ws_bytes, void* stream) {
  Call c;
  digs_status s = prepare(g, lat, phi, w, views, P, opts, nullptr, ws, ws_bytes, stream, c);
  if (s != DIGS_OK) return s;
  if (!meas || !loss_out) return DIGS_ERR_ARG;
  if (P == 0) {
    DIGS_TRY(cudaMemsetAsync(loss_out, 0, sizeof(float), c.st));
    return DIGS_OK;
  }
  s = bin(c, phi, w);
  if (s != DIGS_OK) return s;
  const float inv_count = 1.f / ((float)P * c.ws.nu * c.ws.nv);
  DIGS_TRY(launch_raster_fwd(c.ws, c.views, c.c2, proj, meas, nullptr, inv_count, c.st));
  mark(c, 4);
  DIGS_TRY(launch_loss_reduce(c.ws.loss_part, P * c.ws.T * fwd_blocks(c.ws.tile), loss_out, inv_count, c.st));
  return DIGS_OK;
}

digs_status digs_project_bwd(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                             const DigsView* views, int P, const DigsOpts* opts, const float* grad_proj,
                             float* g_mu0, float* g_scale, float* g_quat, float* g_rho, float* g_phi, float* g_w,
                             void* ws, size_t ws_bytes, void* stream) {
  Call c;
  digs_status s = prepare(g, lat, phi, w, views, P, opts, nullptr, ws, ws_bytes, stream, c);
  if (s != DIGS_OK) return s;
  if (!g_phi || (P > 0 && (!g_w || !grad_proj))) return DIGS_ERR_ARG;
  if (g->n > 0 && (!g_mu0 || !g_scale || !g_quat || !g_rho)) return DIGS_ERR_ARG;
  if (P == 0) {
    DIGS_TRY(cudaMemsetAsync(g_phi, 0, phi_floats(c.L) * 4, c.st));
    if (g->n > 0) {
      DIGS_TRY(cudaMemsetAsync(g_mu0, 0, (size_t)g->n * 12, c.st));
      DIGS_TRY(cudaMemsetAsync(g_scale, 0, (size_t)g->n * 12, c.st));
      DIGS_TRY(cudaMemsetAsync(g_quat, 0, (size_t)g->n * 16, c.st));
      DIGS_TRY(cudaMemsetAsync(g_rho, 0, (size_t)g->n * 4, c.st));
    }
    return DIGS_OK;
  }
  if (!(opts && (opts->flags & DIGS_FLAG_REUSE_BINNING))) {  // else the records of the forward call stand
    s = prep(c, phi, w);
    if (s != DIGS_OK) return s;
  }
  return backward(c, phi, w, grad_proj, g_mu0, g_scale, g_quat, g_rho, g_phi, g_w, P);
}

size_t digs_state_moments(int n, const DigsLattice* lat, int n_w, int n_scans) {
  if (!lat || n < 0 || n_w < 0 || n_scans > DIGS_MAX_SCANS) return 0;
  const size_t S = n_scans > 1 ? (size_t)n_scans : 1;
  return (size_t)n * 11 + S * lat->nx * lat->ny * lat->nz * 3 * lat->R + (size_t)n_w * lat->R;
}

digs_status digs_step(DigsState* st, const float* meas, const int* proj_ids, const DigsView* views, int B,
                      const DigsOpts* opts, float* loss_out, void* ws, size_t ws_bytes, void* stream) {
  if (!st || !meas || !proj_ids || !loss_out || !st->m || !st->v || !st->grad || B < 1) return DIGS_ERR_ARG;
  for (int b = 0; b < B; ++b)
    if (proj_ids[b] < 0 || proj_ids[b] >= st->n_w) return DIGS_ERR_ARG;
  Call c;
  DigsGaussians g{st->n, st->mu0, st->scale, st->quat, st->rho};
  digs_status s = prepare(&g, &st->lat, st->phi, st->w, views, B, opts, proj_ids, ws, ws_bytes, stream, c, st);
  if (s != DIGS_OK) return s;
  const int n = st->n, R = st->lat.R;
  const size_t nphi = c.sc.S * phi_floats(c.L);  // all scans' control points
  float* gr = st->grad;
  float *g_mu0 = gr, *g_ls = gr + 3 * (size_t)n, *g_q = gr + 6 * (size_t)n, *g_rho = gr + 10 * (size_t)n;
  float *g_phi = gr + 11 * (size_t)n, *g_w = g_phi + nphi;
  const bool temporal = st->w_ctrl != nullptr;
  RowsParam rowsp;
  if (temporal) {
    if (c.sc.S > 1 || st->n_ctrl < 1 || !(st->t_step > 0.f)) return DIGS_ERR_ARG;
    for (int b = 0; b < B; ++b) rowsp.v[b] = proj_ids[b];
    DIGS_TRY(launch_temporal_eval(st->w_ctrl, st->n_ctrl, R, st->t_step, rowsp, B, st->w, c.st));
  }
  float* g_w_rows = temporal ? c.ws.gw_rows : g_w;  // dL/dw per row; with control points, their adjoint follows
  s = bin(c, st->phi, st->w);
  if (s != DIGS_OK) return s;
  float inv_count = 1.f / ((float)B * c.ws.nu * c.ws.nv);
  DIGS_TRY(launch_raster_fwd(c.ws, c.views, c.c2, c.ws.proj, meas, c.ws.dldi, inv_count, c.st));
  mark(c, 4);
  DIGS_TRY(launch_loss_reduce(c.ws.loss_part, B * c.ws.T * fwd_blocks(c.ws.tile), loss_out, inv_count, c.st));
  s = backward(c, st->phi, st->w, nullptr, g_mu0, g_ls, g_q, g_rho, g_phi, g_w_rows, st->n_w, st->dens_grad);
  if (s != DIGS_OK) return s;
  if (temporal) DIGS_TRY(launch_temporal_bwd(g_w_rows, st->n_ctrl, R, st->t_step, rowsp, B, g_w, c.st));
  const DigsAdamConfig& a = st->adam;
  float lr[6];
  for (int k = 0; k < 6; ++k) {
    float t = a.total_iters > 1 ? std::min(std::max((float)st->iter / (float)(a.total_iters - 1), 0.f), 1.f) : 0.f;
    lr[k] = a.lr0[k] + (a.lr1[k] - a.lr0[k]) * t;
  }
  size_t sizes[6] = {3 * (size_t)n, 3 * (size_t)n, 4 * (size_t)n, (size_t)n, nphi,
                     temporal ? (size_t)st->n_ctrl * R : (size_t)st->n_w * R};
  float* params[6] = {st->mu0, st->scale, st->quat, st->rho, st->phi, temporal ? st->w_ctrl : st->w};
  const float* grads[6] = {g_mu0, g_ls, g_q, g_rho, g_phi, g_w};
  int kinds[6] = {0, 1, 0, 2, 0, 0};
  AdamGroup groups[6];
  size_t off = 0;
  for (int k = 0; k < 6; ++k) {
    const float lr_k = st->iter_dev ? a.lr0[k] : lr[k];
    groups[k] = AdamGroup{params[k], grads[k], st->m + off, st->v + off, (long long)sizes[k], 0, kinds[k], lr_k,
                          a.lr1[k]};
    off += sizes[k];
  }
  DIGS_TRY(launch_adam(groups, 6, a.beta1, a.beta2, a.eps, st->iter + 1, st->iter_dev, a.total_iters, c.st));
  mark(c, 8);
  if (!st->iter_dev) st->iter += 1;
  return DIGS_OK;
}

digs_status digs_sync_status(void* ws, void* stream) {
  if (!ws) return DIGS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  DIGS_TRY(cudaStreamSynchronize(st));
  DIGS_TRY(cudaMemcpy(&h, ws, sizeof(int), cudaMemcpyDeviceToHost));
  DIGS_TRY(cudaMemset(ws, 0, sizeof(int)));
  return (digs_status)h;
}

digs_status digs_stage_times(float* ms) {
  if (!ms) return DIGS_ERR_ARG;
  for (int i = 0; i < DIGS_NUM_STAGES; ++i) ms[i] = 0.f;
  if (!g_ev_ready || !(g_ev_marked & 1u)) return DIGS_OK;
  int last = 0;
  for (int i = 0; i <= DIGS_NUM_STAGES; ++i)
    if (g_ev_marked & (1u << i)) last = i;
  DIGS_TRY(cudaEventSynchronize(g_ev[last]));
  // stage i spans from boundary i to the next recorded boundary; stage 4 (loss) ends at boundary 5
  int prev = 0;
  for (int i = 1; i <= DIGS_NUM_STAGES; ++i) {
    if (!(g_ev_marked & (1u << i))) continue;
    float t = 0.f;
    DIGS_TRY(cudaEventElapsedTime(&t, g_ev[prev], g_ev[i]));
    ms[i - 1] = t;
    prev = i;
  }
  return DIGS_OK;
}

long long digs_kernel_launches(void) { return g_launches.load(); }

digs_status digs_pair_stats(void* ws, long long* out, void* stream) {
  if (!ws || !out) return DIGS_ERR_ARG;
  Workspace w;
  layout(&w, ws, 0, 0, 1, 1, 1, 0, 16, 0);
  uint32_t np[2] = {0, 0};
  unsigned long long cnt[2] = {0, 0};
  DIGS_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  DIGS_TRY(cudaMemcpy(np, w.n_pairs, sizeof(np), cudaMemcpyDeviceToHost));
  DIGS_TRY(cudaMemcpy(cnt, w.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  out[0] = np[0];
  out[1] = (long long)cnt[0];
  out[2] = (long long)cnt[1];
  return DIGS_OK;
}

const char* digs_status_string(digs_status s) {
  switch (s) {
    case DIGS_OK: return "ok";
    case DIGS_ERR_ARG: return "invalid argument";
    case DIGS_ERR_CUDA: return "CUDA error";
    case DIGS_ERR_CAPACITY: return "workspace too small for the (tile, Gaussian) pairs";
    case DIGS_ERR_TIMEOUT: return "device-side wait timed out";
    case DIGS_ERR_NONFINITE: return "non-finite input";
  }
  return "unknown status";
}

}  // extern "C"
