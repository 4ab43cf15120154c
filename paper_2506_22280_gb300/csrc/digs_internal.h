// Host-side launchers shared between the translation units of libdigs (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "digs_common.cuh"

namespace digs {

// Kernel-launch bookkeeping (diagnostic): every launcher reports how many kernels it enqueued.
void note_launches(int k);

// Workspace carve-up for one call.  Every pointer is 256-byte aligned inside the caller's buffer.
struct Workspace {
  int* status;            // [4]  device-detected status
  uint32_t* n_pairs;      // [2]  number of (tile, Gaussian) pairs produced, pairs kept (<= cap)
  unsigned long long* counters;  // [2] forward raster: box pairs evaluated, pairs within the cutoff
  float4* rec;            // [P * n * 3]
  uint32_t* counts;       // [P * n + 1] tiles touched per (projection, Gaussian)
  uint2* tbox;            // [P * n] tile rectangle of each record: (tx0 | ty0 << 16, tx1 | ty1 << 16)
  uint32_t* chist;        // [P * T * chunks + 1] direct binning: pairs per (projection, tile, record chunk), then their scan
  uint32_t* offsets;      // [P * n + 1] exclusive scan of counts (offsets[P*n] = total)
  uint32_t* scan_tmp;     // block sums of the scans
  uint32_t* keys;         // [cap] (projection, tile) key per pair
  uint32_t* vals;         // [cap] (projection, Gaussian) record of the pair
  uint32_t* keys_alt;     // [cap]
  uint32_t* vals_alt;     // [cap]
  uint32_t* srid;         // record of each sorted position (the sorted values: vals or vals_alt)
  uint32_t* hist;         // radix histograms [256][sort blocks]
  uint32_t* seg;          // [2P + 2] each projection's first pair and first sort block
  uint2* ranges;          // [P * T] sorted-range of each (projection, tile)
  uint32_t* order;        // [P * T] forward launch order (longest lists first)
  float4* grec;           // [P * n * 3] backward: the ten pixel sums of each (projection, Gaussian) record
  uint8_t* bcost;         // [P * n] backward sweep cost of each record: box pixels / 32, capped at 255
  uint8_t* bperm;         // [P][32 ceil(n / 32)] backward: each group of 32 records in order of sweep cost
  float* gw_part;         // [pair-sum CTAs][P][R] dL/dw partial sums
  float* ffd;             // [12 R][n_total]: u_r (3R components) then grad u_r (9R) at each mean
  float* ffd2;            // [18 R][n_total]: second derivatives of u_r (6 per component)
  float* gsum;            // [11 + 12 R][n_total]: each Gaussian's pair adjoints summed over its projections
  float* loss_part;       // [P * T * fwd_blocks(tile)] forward: squared residuals per 8 x 8 block (warp)
  float* proj;            // [P * nv * nu] (digs_step)
  float* dldi;            // [P * nv * nu] (digs_step)
  float* gw_rows;         // [w rows][R] (digs_step with temporal control points): dL/dw before the adjoint
  float* grads;           // all parameter gradients (digs_step)
  size_t bytes;
  long long cap;
  int n, P, nu, nv, R, tile, tiles_x, tiles_y, T;  // n: record stride (largest scan's Gaussian count)
  int n_total;                                     // Gaussians of all scans
  int bwd_lanes;                                   // lanes per record in the backward raster (16 or 32)
  int n_sort_blocks;
  int n_chunks;                                    // record chunks of the direct binning (-1: radix-sort path)
};

// Forward work items (8 x 8 pixel blocks) per tile.
inline int fwd_blocks(int tile) { return (tile / 8) * (tile / 8); }

size_t layout(Workspace* ws, void* base, int n, int P, int nu, int nv, int R, long long cap, int tile, int n_total,
              int w_rows = 0);

// scan.cu
cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int n, uint32_t* tmp, cudaStream_t st);
size_t scan_tmp_words(int n);

// sort.cu: stable sort of the pair keys (projection * T + tile) with their record values, the pairs being
// grouped by projection as the emit step writes them (projection b's start is offsets[b * n]); count
// read from the device; also writes ranges[P * T].  Returns via *out_keys / *out_vals which of the two
// buffers holds the result (*out_keys = nullptr after a single pass, T <= 256: the sorted keys are then
// not written, only the ranges are needed).  seg: 2P + 2 words; hist: 256 * n_blocks + 1 words, n_blocks = sort_blocks.
cudaError_t sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, const uint32_t* n_dev,
                       long long cap, const uint32_t* offsets, int n, int P, int T, int n_blocks, uint32_t* seg,
                       uint32_t* hist, uint32_t* scan_tmp, uint2* ranges, uint32_t** out_keys, uint32_t** out_vals,
                       cudaStream_t st);
// Per-(projection, tile) ranges of the sorted keys.
cudaError_t tile_ranges(const uint32_t* sorted_keys, const uint32_t* n_dev, long long cap, uint2* ranges,
                        int n_ranges, cudaStream_t st);
int sort_blocks(long long cap, int P);
// Direct binning (T <= kDirectMaxTiles): counting sort of the (projection, tile) pairs straight from the
// records' tile rectangles into ws.vals, plus ranges, pair counts and the capacity flag.
constexpr int kDirectMaxTiles = 1024;
int bin_chunks(int n, int T);
cudaError_t bin_direct(const Workspace& ws, cudaStream_t st);
// order[P * T]: (projection, tile) indices by descending range length (power-of-two classes).
cudaError_t tile_order(const uint2* ranges, int n, uint32_t* order, cudaStream_t st);

// prep.cu
cudaError_t launch_ffd_eval(const LatticeC& L, const float* phi, const float* x, int n, float* U, float* dU,
                            cudaStream_t st);
cudaError_t launch_prep_fwd(const GaussPtrs& g, const ScanTable& sc, const LatticeC& L, const float* phi,
                            const float* w, const ViewsParam& views, int P, float c2, const Workspace& ws,
                            cudaStream_t st);
cudaError_t launch_emit(const Workspace& ws, cudaStream_t st);

// raster.cu
cudaError_t launch_raster_fwd(const Workspace& ws, const ViewsParam& views, float c2, float* proj, const float* meas,
                              float* dldi, float inv_count, cudaStream_t st);
// grad_proj = dL/dI, or nullptr when ws.dldi already holds dL/dI * |X - s| (from the step's forward).
cudaError_t launch_raster_bwd(const Workspace& ws, const ViewsParam& views, float c2, const float* grad_proj,
                              cudaStream_t st);
// Sums part[0 .. n) in a fixed order (overwriting part) and writes scale * sum to out[0].
cudaError_t launch_loss_reduce(float* part, int n, float* out, float scale, cudaStream_t st);

// chain.cu
cudaError_t launch_chain_bwd(const GaussPtrs& g, const ScanTable& sc, const LatticeC& L, const float* phi,
                             const float* w, const ViewsParam& views, int P, const Workspace& ws, float* g_mu0,
                             float* g_scale, float* g_quat, float* g_rho, float* g_phi, float* dens_grad,
                             cudaStream_t st);
cudaError_t launch_gw_reduce(const Workspace& ws, const ViewsParam& views, int P, int R, float* g_w, int w_rows,
                             cudaStream_t st);
int chain_blocks(int n);
int pair_sum_blocks(int n);

// umma.cu: tensor-core GEMM behind digs_gemm_bf16 (BF16 operands rounded from FP32, FP32 accumulation); C(m, n) = sum_k
// A(m, k) B(k, n) with A(m, k) = at ? A[k lda + m] : A[m lda + k], B(k, n) = bt ? B[n ldb + k] :
// B[k ldb + n]; splits > 1: partial sums over K ranges into C + z zstride (bias and ReLU not applied).
// *status (optional) is set to 1 if a bounded wait gave up.
cudaError_t gemm_tc(bool at, bool bt, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                    int ldc, const float* bias, bool relu, int splits, long long zstride, int* status,
                    cudaStream_t st);
// The same with the K splits (splits > 1) summed in order into C by a second kernel, adding the bias and
// applying ReLU there; part: splits * M * N floats.
cudaError_t gemm_tc_sum(bool at, bool bt, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                        float* C, int ldc, const float* bias, bool relu, int splits, float* part, int* status,
                        cudaStream_t st);

// temporal.cu: w rows of a step from the temporal B-spline control points, and the adjoint.
struct RowsParam {
  int v[DIGS_MAX_VIEWS];
};
cudaError_t launch_temporal_eval(const float* ctrl, int n_ctrl, int R, float t_step, const RowsParam& rows, int B,
                                 float* w, cudaStream_t st);
cudaError_t launch_temporal_bwd(const float* g_w, int n_ctrl, int R, float t_step, const RowsParam& rows, int B,
                                float* g_ctrl, cudaStream_t st);

// cnn_tc.cu: the weight-predictor CNN on the tensor cores.  Parameter and gradient pointers per layer
// (FP32, in cnn.cu's layout: conv weights [Co][3][3][Ci], dense weights W1 [128][8194]).
struct CnnNet {
  const float *w[4], *b[4], *w1, *b1;
};
struct CnnGrad {
  float *w[4], *b[4], *w1;
};
// BF16 (16-bit words) and FP32 buffers of one batch size, carved out of the caller's workspace.
struct CnnTc {
  uint16_t *imgb, *act[3], *feat, *dy[2], *dy3, *dhb, *wb[4], *w1b, *wt[4];
  float *part, *colpart;
  long long part_floats, colpart_floats;
  unsigned* tickets;  // counters of the single-launch column reductions (zeroed by cnn_tc_backward)
};
// Bytes of the buffers for batch B (base == nullptr: size only), 256-byte aligned.
size_t cnn_tc_layout(void* base, int B, CnnTc* t);
// Forward to the dense layer's ReLU output h [B][128] (FP32); keeps the activations for the backward.
cudaError_t cnn_tc_forward(const CnnNet& net, const float* img, const float* cs, int B, const CnnTc& t, float* h,
                           cudaStream_t st);
// Parameter gradients of every layer but the output one (and but the dense layer's bias), from
// dh = dL/d(dense pre-activation) [B][128] (already masked by the dense layer's ReLU; its BF16 copy in
// t.dhb, written by the caller with it), through the activations and weights that the last
// cnn_tc_forward on the same buffers kept.
cudaError_t cnn_tc_backward(int B, const CnnTc& t, const float* dh, const CnnGrad& g, cudaStream_t st);

// adam.cu
struct AdamGroup {
  float* p;
  const float* g;
  float* m;
  float* v;
  long long n;
  long long off;   // offset of this group inside m / v
  int kind;        // 0 plain, 1 log-parameterised (scale), 2 softplus-parameterised (density)
  float lr;        // learning rate of this step, or (iter_dev set) of step 0
  float lr_end;    // (iter_dev set) learning rate of step total_iters - 1, linear in between
};
// step: 1-based Adam step (bias correction) when iter_dev is null; else the step count is read from
// *iter_dev (0-based) on the device and a following kernel increments it.
cudaError_t launch_adam(const AdamGroup* groups, int ngroups, float beta1, float beta2, float eps, int step,
                        int* iter_dev, int total_iters, cudaStream_t st);

}  // namespace digs
