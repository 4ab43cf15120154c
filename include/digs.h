/*
 * digs.h -- C-ABI of the GB300 (sm_103a) DIGS hot path.
 *
 * DIGS (arXiv 2506.22280) reconstructs dynamic cone-beam CT as a cloud of 3D Gaussians warped by a
 * low-rank cubic B-spline free-form deformation (FFD).  For every projection the hot path evaluates the
 * FFD and its Jacobian at each Gaussian mean (Sec. 3.3, Eq. 9-11), moves the mean and transforms the
 * covariance Sigma' = K Sigma K^T (Sec. 3.2, Eq. 7-8), integrates every deformed Gaussian along every
 * detector ray in closed form (the X-ray transform of Sec. 3.1, Eq. 1-4), and runs the backward pass of
 * a projection-domain L2 loss (Sec. 4.2).
 *
 * Conventions shared by every entry point:
 *  - All array pointers are DEVICE pointers to contiguous FP32 (or int32) memory owned by the caller,
 *    unless a comment says "host".  The library allocates no memory: scratch space is a caller-owned
 *    workspace of digs_workspace_size() bytes.
 *  - Calls are enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and return without
 *    synchronising, except digs_count_pairs() and digs_sync_status(), which say so.
 *  - Host-detected errors (bad arguments, launch failures) are returned at once.  Device-detected errors
 *    (workspace too small for the number of (ray-tile, Gaussian) pairs) are recorded in a status word
 *    inside the workspace; digs_sync_status() reports and clears it.
 *  - Gradient outputs are overwritten, never accumulated into.
 *
 * Layouts (N Gaussians, P projections, R <= DIGS_MAX_R ranks):
 *  mu0[N][3] mm, scale[N][3] mm (> 0), quat[N][4] as (w, x, y, z) (normalised inside), rho[N] mm^-1:
 *      the reference Gaussians, Sigma = R(q) diag(scale)^2 R(q)^T (Sec. 3.1, after Eq. 2).
 *  phi[R][nz][ny][nx][3] mm: control-point displacements d^r_ijk (Sec. 3.3, Eq. 10); node (i, j, k)
 *      sits at origin + (i, j, k) * spacing, i (x) fastest.  Nodes outside the lattice read as zero.
 *  w[P][R]: temporal weights omega_r(t) at each projection's time point (Eq. 9).
 *  proj[P][nv][nu]: line integrals, pixel (i, j) at proj[p][j][i].
 */
#ifndef DIGS_H
#define DIGS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIGS_MAX_R 4        /* ranks N_r of the low-rank motion model (the paper uses 2)            */
#define DIGS_MAX_VIEWS 128  /* projections per call                                                 */
#define DIGS_MAX_SCANS 8    /* independent scans rendered together by one digs_step call             */

typedef enum {
  DIGS_OK = 0,
  DIGS_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, non-finite geometry, ...)    */
  DIGS_ERR_CUDA = 2,       /* a CUDA launch or runtime call failed                                   */
  DIGS_ERR_CAPACITY = 3,   /* more (tile, Gaussian) pairs than the workspace holds: grow and retry   */
  DIGS_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up                                     */
  DIGS_ERR_NONFINITE = 5   /* a non-finite value was found where finite input was required           */
} digs_status;

/* Reference Gaussians {rho_n, mu_n, R_n, S_n} (Sec. 3.1, Eq. 2).  n may be 0. */
typedef struct {
  int n;
  const float* mu0;    /* [n][3] */
  const float* scale;  /* [n][3] */
  const float* quat;   /* [n][4] (w, x, y, z) */
  const float* rho;    /* [n]    */
} DigsGaussians;

/* Uniform control lattice of the FFD spatial basis (Sec. 3.3, text before Eq. 10). */
typedef struct {
  int nx, ny, nz, R;
  float origin[3];   /* world position of node (0, 0, 0), mm */
  float spacing[3];  /* node spacing per axis, mm (> 0)      */
} DigsLattice;

/* One projection's scan geometry (host memory, double precision).  The detector axes e_u, e_v must be
 * orthonormal.  Pixel (i, j) has centre det_c + (i - (nu-1)/2 + off_u) du e_u + (j - (nv-1)/2 + off_v) dv e_v.
 * Cone beam (parallel = 0): rays run from src through each pixel centre.  Parallel beam: rays run
 * through each pixel centre along the unit vector from src to det_c. */
typedef struct {
  double src[3], det_c[3], e_u[3], e_v[3];
  double du, dv, off_u, off_v;
  int nu, nv, parallel;
  int scan;          /* digs_step: which scan of the state this projection belongs to (0 otherwise) */
} DigsView;

/* Options.  cutoff: a (ray, Gaussian) pair contributes iff the squared Mahalanobis distance E from the
 * ray to the deformed mean is <= cutoff^2 (default 3.5).  tile: square raster tile edge in pixels (8, 16
 * or 32; 0 = 16).  flags: DIGS_FLAG_* bits.  bwd_lanes: lanes that share one (projection, Gaussian) pair
 * in the backward raster, 16 (two Gaussians per warp) or 32 (one); 0 = 16.  Tile and lanes change the
 * speed, not the result beyond rounding. */
typedef struct {
  float cutoff;
  int tile;
  int flags;
  int bwd_lanes;
} DigsOpts;

#define DIGS_FLAG_EWA 4            /* cone-beam views: the paper's 2D-Gaussian approximation of each projected
                                      Gaussian (Sec. 3.1, Eq. 4: EWA covariance of J W Sigma W^T J^T with
                                      its third row and column dropped, density scaled by the integration
                                      bias factor) instead of the exact line integral; a pair contributes
                                      where its 2D Mahalanobis distance is <= cutoff.  Parallel views are
                                      exact either way (the two models coincide there).               */
#define DIGS_FLAG_REUSE_BINNING 1  /* project_bwd: reuse the per-pair records left in `ws` (same size)
                                      by the immediately preceding project_fwd with identical inputs   */

/* Bytes of workspace for n Gaussians, P projections of nu x nv pixels, R ranks and room for
 * `max_pairs` (tile, Gaussian) pairs.  Use digs_count_pairs() to learn the pair count of an input. */
size_t digs_workspace_size(int n, int P, int nu, int nv, int R, long long max_pairs, const DigsOpts* opts);

/* u_r(x) and its world-space gradient at each point (Sec. 3.3, Eq. 10 and the gradient inside Eq. 11).
 * x[n][3] in; U[n][R][3] and dU[n][R][3][3] out, dU[.][r][i][j] = d u_{r,i} / d x_j.
 * One thread per point; needs no workspace. */
digs_status digs_ffd_eval(const DigsLattice* lat, const float* phi, const float* x, int n,
                          float* U, float* dU, void* stream);

/* Number of (tile, Gaussian) pairs the binning of these inputs produces, written to *count_host.
 * SYNCHRONISES the stream.  `ws` may be sized with max_pairs = 0. */
digs_status digs_count_pairs(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                             const DigsView* views, int P, const DigsOpts* opts, void* ws, size_t ws_bytes,
                             long long* count_host, void* stream);

/* Forward projection: deform the Gaussians at each projection's weights (Eq. 7-11) and integrate them
 * along every detector ray (Eq. 1, 3, 4), writing proj[P][nv][nu].  All views in one call must share
 * nu and nv.  views: host array [P]. */
digs_status digs_project_fwd(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                             const DigsView* views, int P, const DigsOpts* opts, float* proj,
                             void* ws, size_t ws_bytes, void* stream);

/* Forward projection without a workspace (the paper has no counterpart to this entry point; it exists
 * for callers).  Same inputs, output and result as digs_project_fwd, but its scratch memory is a
 * file-scope device array of DIGS_STATIC_SCRATCH_BYTES (32 MiB) inside this library, so the caller
 * allocates nothing.  It serves callers that cannot call cudaMalloc: plug-ins whose host application
 * owns all device memory through its own allocator, code that runs under a fixed device-memory budget
 * set before it is loaded, and small C programs that should not have to size and manage a workspace.
 *  - Every GPU on which the library's device code is loaded holds the 32 MiB until the process exits.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 *    device current.
 *  - Synchronous: the call waits for its stream and returns the status the device recorded.  It cannot
 *    be used inside stream capture (it reads that status back to the host) and returns DIGS_ERR_ARG,
 *    launching nothing, when `stream` is capturing.
 *  - All calls share the array and each overwrites what the last one left: calls whose work overlaps
 *    on the GPU (other streams, other host threads) race and must not be issued.
 *  - Returns DIGS_ERR_ARG, before launching anything, when the problem's pair-independent scratch,
 *    digs_workspace_size(n, P, nu, nv, R, 0, opts) bytes (about 118 B per (projection, Gaussian) +
 *    (168 R + 68) B per Gaussian + 8 B per pixel), exceeds the array.  Returns DIGS_ERR_CAPACITY if the
 *    (tile, Gaussian) pairs (16 B each) did not fit in the rest of the array; the output is then
 *    incomplete, and the next call starts with a clear status.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine. */
#define DIGS_STATIC_SCRATCH_BYTES (32u << 20)
digs_status digs_project_fwd_static(const DigsGaussians* g, const DigsLattice* lat, const float* phi,
                                    const float* w, const DigsView* views, int P, const DigsOpts* opts,
                                    float* proj, void* stream);

/* Forward projection and the L2 projection loss of Sec. 4.2 in one pass: writes
 * loss_out[0] (device float) = mean over the P nv nu pixels of (I - meas)^2, with I the projections of
 * digs_project_fwd; the residuals are squared and summed inside the raster kernel (per 8 x 8 block, then
 * added in a fixed order), so no image needs to be read back.  meas: [P][nv][nu]; proj: optional
 * [P][nv][nu] output of I (NULL: not written).  Same workspace as digs_project_fwd. */
digs_status digs_project_loss(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                              const DigsView* views, int P, const DigsOpts* opts, const float* meas, float* proj,
                              float* loss_out, void* ws, size_t ws_bytes, void* stream);

/* Backward projection: given grad_proj = dL/dproj [P][nv][nu], write dL/d of every input:
 * g_mu0[n][3], g_scale[n][3], g_quat[n][4], g_rho[n], g_phi[R][nz][ny][nx][3], g_w[P][R].
 * The truncated sum is differentiated almost everywhere (the cutoff's boundary term is ignored).
 * Needs no tile lists: `ws` may be sized with max_pairs = 0. */
digs_status digs_project_bwd(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                             const DigsView* views, int P, const DigsOpts* opts, const float* grad_proj,
                             float* g_mu0, float* g_scale, float* g_quat, float* g_rho, float* g_phi, float* g_w,
                             void* ws, size_t ws_bytes, void* stream);

/* Adam hyper-parameters of one reconstruction (Sec. 4.2: Adam, learning rates decaying linearly from
 * lr0 to lr1 over total_iters).  Groups: means (mm), log-scales, quaternions, density pre-activation
 * (rho = softplus(theta)), the spatial B-spline grid phi and the temporal weights w. */
typedef struct {
  float lr0[6], lr1[6];   /* per group: mu0, log-scale, quat, density, phi, w */
  float beta1, beta2, eps;
  int total_iters;
} DigsAdamConfig;

/* Reconstruction state in caller-owned device memory.  Parameters are updated in place.  m and v are
 * Adam moments laid out like the parameters, concatenated in group order
 * (mu0 3n, log-scale 3n, quat 4n, density n, phi S*R*nz*ny*nx*3, w n_w*R), zero before the first step.
 * Several independent scans (S = n_scans <= DIGS_MAX_SCANS, e.g. scans of different patients with uneven
 * Gaussian counts) may share one state so that one digs_step renders projections of all of them in one
 * launch per stage: scan s owns Gaussians [scan_off[s], scan_off[s+1]) (scan_off[0] = 0,
 * scan_off[S] = n), control points phi[s] ([S][R][nz][ny][nx][3], one lattice geometry for all scans),
 * and the rows of w that its projections name; each view passed to digs_step says its scan.
 * n_scans <= 1 means one scan holding all n Gaussians (scan_off is then ignored). */
typedef struct {
  int n;
  float *mu0, *scale, *quat, *rho;  /* physical parameters (scale > 0, rho > 0)     */
  float *phi;                        /* [S][R][nz][ny][nx][3]                        */
  float *w;                          /* [n_w][R]: weights of every time point of the scan */
  int n_w;
  float *m, *v;                      /* Adam moments                                 */
  float *grad;                       /* gradient scratch, laid out like m            */
  int iter;                          /* completed steps; digs_step increments it     */
  DigsLattice lat;
  DigsAdamConfig adam;
  int n_scans;
  int scan_off[DIGS_MAX_SCANS + 1];
  int* iter_dev;                     /* optional device int: when set, the step count (learning-rate
                                        schedule, Adam bias correction) is read from and incremented on
                                        the device, so a captured CUDA graph of a step can be replayed;
                                        `iter` is then neither read nor changed                        */
  float* w_ctrl;                     /* optional [n_ctrl][R]: temporal B-spline control points of the
                                        weights (Sec. 4.2; one scan only).  When set, each step first
                                        writes the rows proj_ids of w from them -- projection p at
                                        tau = p / t_step + 1 control-point units, f = floor(tau) - 1,
                                        u = tau - floor(tau), w(p) = sum_l B_l(u) w_ctrl[f + l], outside
                                        nodes zero -- and Adam updates w_ctrl instead of w (the last
                                        group of m / v / grad is then n_ctrl * R floats)              */
  int n_ctrl;
  float t_step;                      /* control-point spacing in projection indices (e.g. 4)          */
  float* dens_grad;                  /* optional [n]: when set, each step adds, for every Gaussian, the
                                        sum over the batch's projections of |dL/dmu'_b| (the gradient of
                                        the step's loss with respect to its deformed mean in projection b,
                                        the deformed covariance held fixed): the statistic of
                                        digs_densify_plan.  Single-scan states only.                    */
} DigsState;

/* Number of floats in DigsState.m (and v, grad) for n Gaussians in n_scans (>= 1) scans with per-row
 * weights w (for temporal control points use digs_state_size). */
size_t digs_state_moments(int n, const DigsLattice* lat, int n_w, int n_scans);

/* Number of floats in m (and v, grad) for the state as configured (scans, temporal control points). */
size_t digs_state_size(const DigsState* st);

/* Bytes of workspace digs_step needs for the state's scans, B projections of nu x nv pixels and room for
 * max_pairs (tile, Gaussian) pairs (records are laid out [B][largest scan's Gaussian count]). */
size_t digs_state_workspace_size(const DigsState* st, int B, int nu, int nv, long long max_pairs,
                                 const DigsOpts* opts);

/* One optimisation step over a batch of B projections (Eq. 1 with the L2 loss of Sec. 4.2):
 * render the projections `proj_ids` (host int array [B], rows of st->w) with geometry views[B] (host),
 * loss = mean over the batch's pixels of (I - meas)^2 written to loss_out (device float), gradients of
 * every parameter, then one fused Adam update of all groups with the learning rates of iteration st->iter.
 * meas: [B][nv][nu].  views[b].scan names the scan projection b belongs to (all 0 for one scan); every
 * stage is one launch over all B projections of all scans.  The workspace must be sized by
 * digs_state_workspace_size (for one scan, digs_workspace_size with n Gaussians and B projections). */
digs_status digs_step(DigsState* st, const float* meas, const int* proj_ids, const DigsView* views, int B,
                      const DigsOpts* opts, float* loss_out, void* ws, size_t ws_bytes, void* stream);

/* Synchronise `stream`, return the device-detected status recorded in `ws` since the last call, and
 * clear it. */
digs_status digs_sync_status(void* ws, void* stream);

/* ---- Evaluation volumes at one time point ------------------------------------------------------ */

/* Voxel grid: centre of voxel (i, j, k) = origin + (i, j, k) * spacing (mm), i (x) fastest. */
typedef struct {
  int nx, ny, nz;
  float origin[3], spacing[3];
} DigsGrid;

/* Attenuation volume of the cloud deformed with the weights w[R] of one time point (Eq. 3 with the warp
 * of Eq. 7-8): vol[nz][ny][nx] = sum_n rho_n exp(-E_n / 2) at the voxel centres, E_n the squared
 * Mahalanobis distance to the deformed mean, each Gaussian taken where E_n <= cutoff^2 (opts->cutoff,
 * default 3.5); folded Gaussians (det K <= 1e-6) are dropped.  Sums use float atomics, so the result
 * varies between runs within rounding.  w: device [R]. */
digs_status digs_voxelize(const DigsGaussians* g, const DigsLattice* lat, const float* phi, const float* w,
                          const DigsGrid* grid, const DigsOpts* opts, float* vol, void* stream);

/* Displacement field of one time point, D(x, t) - x = sum_r w_r u_r(x) (Eq. 9-10), at the voxel centres:
 * dvf[nz][ny][nx][3] mm.  w: device [R]. */
digs_status digs_dvf(const DigsLattice* lat, const float* phi, const float* w, const DigsGrid* grid, float* dvf,
                     void* stream);

/* ---- Weight-predictor CNN (warm start of the temporal weights) ---------------------------------
 * The paper has no counterpart: this network learns, from (projection, weights) pairs that the forward
 * model above renders, to map one projection to its R temporal weights, so that a reconstruction can
 * start its per-projection weights near their values.  Input: the projection 2x2-averaged to 128 x 128
 * (digs_cnn_prepare_input) and (cos theta, sin theta) of its gantry angle; four 3x3 stride-2 convolutions
 * (1 -> 32 -> 64 -> 128 -> 128 channels, ReLU), a 128-unit ReLU layer, a linear layer to R outputs.
 * Parameters: one FP32 array of digs_cnn_params(R) floats, in this order per layer: conv weights
 * [Co][3][3][Ci] and biases [Co] for the four convolutions, then W1 [128][8194] (the 8 x 8 x 128
 * features in (y, x, c) order, then cos, sin), b1 [128], W2 [R][128], b2 [R].  Images: [B][128][128];
 * angle features cs: [B][2]; weights: [B][R].  B <= 1024.  The workspace (digs_cnn_workspace_size)
 * holds the activations of the last forward, which digs_cnn_backward differentiates. */
size_t digs_cnn_params(int R);
size_t digs_cnn_workspace_size(int B, int R);
/* He-normal weights (std sqrt(2 / fan-in)) from a counter-based generator of `seed`; zero biases. */
digs_status digs_cnn_init(float* params, int R, unsigned long long seed, void* stream);
/* img[b] = scale * the 2x2 means of proj[b] ([B][256][256] -> [B][128][128]), or scale * proj[b] for
 * [B][128][128] projections (a detector of half the pixels at twice the pitch). */
digs_status digs_cnn_prepare_input(const float* proj, int B, int nu, int nv, float scale, float* img, void* stream);
/* flags of the forward, backward and training step: DIGS_CNN_TENSOR_CORES runs the convolutions' and the
 * 8194-wide layer's GEMMs on the tensor cores (BF16 operands rounded from FP32, FP32 accumulation); without
 * it every GEMM is FP32 on the SIMT pipes. */
#define DIGS_CNN_TENSOR_CORES 1
/* Forward: w_out[B][R]. */
digs_status digs_cnn_forward(const float* params, int R, const float* img, const float* cs, int B, float* w_out,
                             int flags, void* ws, size_t ws_bytes, void* stream);
/* Gradient of every parameter (grad_params, laid out like params) for dL/dw = grad_w [B][R], through the
 * activations of the preceding digs_cnn_forward on the same workspace and batch size. */
digs_status digs_cnn_backward(const float* params, int R, int B, const float* grad_w, float* grad_params, int flags,
                              void* ws, size_t ws_bytes, void* stream);
/* One training step on the mean squared error between the predicted and target weights ([B][R]):
 * forward, loss (device float, written to loss_out), backward into grad, Adam (beta 0.9 / 0.999,
 * eps 1e-8, learning rate lr, 1-based step) on params with moments m, v (zero-initialised). */
digs_status digs_cnn_train_step(float* params, float* m, float* v, float* grad, int step, float lr, int R,
                                const float* img, const float* cs, const float* target, int B, float* loss_out,
                                int flags, void* ws, size_t ws_bytes, void* stream);
/* Inference with BF16 weights and activations, the large GEMMs on the tensor cores with FP32 accumulation
 * (biases and the output layer FP32): w_out[B][R]. */
digs_status digs_cnn_infer_bf16(const float* params, int R, const float* img, const float* cs, int B, float* w_out,
                                void* ws, size_t ws_bytes, void* stream);

/* ---- Adaptive density control -----------------------------------------------------------------
 * Between optimisation steps the cloud is densified and pruned (Sec. 4.2 gives the gradient threshold,
 * 5e-8 in its loss units, and defers the other settings to the method it builds on, whose values are not
 * stated; the rules below are this library's reading, each a parameter).  Per Gaussian, with g = the
 * DigsState.dens_grad sum over the n_projections projections rendered since it was last cleared:
 *   prune if rho < rho_min; else, if g >= tau * n_projections (compared in float: the product is
 *   rounded to float once), split if the largest scale exceeds s_split, otherwise clone; else keep.
 * Clone: two copies, each with density rho / 2.  Split: two children at mu + R diag(s) z_k (z_k ~ N(0, I)
 * drawn by the caller, z[n][2][3]) with scales s / 1.6, the parent's rotation and density
 * rho * 1.6^3 / 2 (the integrated mass is conserved).  Output rows follow the parents' order, a clone's
 * original first; src[j] is each output row's parent and is_new[j] marks the rows that are not the parent
 * itself (the clone's second copy, both split children), whose optimiser moments should start at zero
 * (digs_gather_rows). */
typedef struct {
  float tau;          /* threshold on the mean of |dL/dmu'| over the projections (paper: 5e-8)   */
  int n_projections;  /* projections rendered since dens_grad was cleared (>= 1)                   */
  float s_split;      /* largest scale above which a densified Gaussian is split (mm)              */
  float rho_min;      /* density below which a Gaussian is pruned                                  */
} DigsDensifyOpts;
size_t digs_densify_workspace_size(int n);
/* action[n]: -1 prune, 0 keep, 1 clone, 2 split; dst[n + 1] (device ints): each Gaussian's first output
 * row, dst[n] = the number of output rows. */
digs_status digs_densify_plan(int n, const float* grad_sum, const float* scale, const float* rho,
                              const DigsDensifyOpts* opts, int* action, int* dst, void* ws, size_t ws_bytes,
                              void* stream);
/* Writes the new cloud (rows [0, dst[n]) of mu0 [.][3], scale [.][3], quat [.][4], rho, src, is_new;
 * rows at or beyond cap are not written).  z: device [n][2][3]. */
digs_status digs_densify_apply(const DigsGaussians* g, const int* action, const int* dst, const float* z, int cap,
                               float* mu0, float* scale, float* quat, float* rho, int* src, int* is_new,
                               void* stream);
/* out[j][c] = is_new[j] ? 0 : in[src[j]][c] for j < n_out, c < dim (e.g. Adam moments of the new cloud). */
digs_status digs_gather_rows(const int* src, const int* is_new, int n_out, int dim, const float* in, float* out,
                             void* stream);

/* ---- Dense GEMM on the tensor cores ------------------------------------------------------------
 * The paper has no counterpart: the weight-predictor CNN's layers run on this.  C = op(A) op(B) (+ bias
 * per column, ReLU if relu != 0) on the fifth-generation tensor cores: A and B are FP32 in device memory,
 * rounded to BF16 (round to nearest even) as they are read; products are exact and accumulate in FP32.
 * op(A) is M x K: A[m lda + k], or A[k lda + m] if trans_a; op(B) is K x N: B[k ldb + n], or
 * B[n ldb + k] if trans_b; C is M x N with row pitch ldc (FP32).  splits > 1 (<= 64) divides K into
 * that many ranges computed in parallel into partial[splits][M][N] (device scratch the caller owns),
 * then added in a fixed order.  status: optional device int set to 1 if an internal bounded wait gave
 * up (the output is then undefined).  DIGS_ERR_ARG on bad sizes or pitches. */
digs_status digs_gemm_bf16(int trans_a, int trans_b, int M, int N, int K, const float* A, int lda, const float* B,
                           int ldb, const float* bias, int relu, float* C, int ldc, int splits, float* partial,
                           int* status, void* stream);

/* Tests each K-loop wait of digs_gemm_bf16's kernel makes on its mbarrier before it gives up (the
 * wait then sets *status to 1 and the output is undefined); tests < 0 restores the default (about
 * 4 x 10^6 tests, well under a second).  The final wait for the block's own tensor-core operations,
 * before it frees its tensor memory, always uses the default.  Process-wide; read when a GEMM is
 * launched (a captured graph keeps the value of its capture).  For testing the give-up path. */
digs_status digs_set_wait_limit(long long tests);

/* ---- Diagnostics (not part of the method; used to measure it) ---------------------------------- */

/* Stage timing: a call whose opts->flags has DIGS_FLAG_TIME_STAGES records CUDA events around each of
 * its stages on its stream.  digs_stage_times() waits for the last of them and writes the milliseconds
 * of each stage of the most recent timed call to ms[DIGS_NUM_STAGES] (0 for stages it did not run):
 * 0 FFD + deformation + projection set-up, 1 binning (per-chunk tile counts, their prefix sum, the
 * record-id scatter and the tile ranges; beyond 1024 tiles per projection: prefix sum + key emission),
 * 2 forward launch order (beyond 1024 tiles: radix sort + tile ranges + launch order), 3 forward raster, 4 loss reduction, 5 backward raster, 6 per-Gaussian chain + FFD backward + dL/dw,
 * 7 fused Adam.  Process-wide state: time one call at a time. */
#define DIGS_FLAG_TIME_STAGES 2
#define DIGS_NUM_STAGES 8
digs_status digs_stage_times(float* ms);

/* Microbenchmark of one arithmetic pipe, for the roofline of the splat kernels (their work per (pixel,
 * Gaussian) pair is FP32 FMA-pipe arithmetic plus two SFU functions).  Enqueues on `stream` one launch
 * of two 1024-thread CTAs per SM whose threads run eight independent chains of `iters` x 4 results (x 8
 * for kind 1) of kind 0: scalar fma.rn.f32, 1: packed fma.rn.f32x2 (two results per instruction), 2: ex2.approx.ftz.f32,
 * 3: rsqrt.approx.ftz.f32, and writes the number of FP32 results of the launch (an FMA counts once) to
 * *lane_ops (host).  Time the launch with CUDA events on the stream; results / time is the pipe's rate.
 * sink: device float the kernel may write (it never does in practice).  Asynchronous. */
digs_status digs_pipe_bench(int kind, int iters, float* sink, long long* lane_ops, void* stream);

/* Number of CUDA kernels this library has launched since it was loaded (memsets not counted). */
long long digs_kernel_launches(void);

/* Pair statistics of the most recent forward pass that used `ws` (synchronises `stream`):
 * out[0] = (tile, Gaussian) pairs binned, out[1] = (pixel, Gaussian) pairs inside the pixel boxes that
 * the forward raster evaluated, out[2] = pairs within the cutoff (E <= cutoff^2) that it accumulated. */
digs_status digs_pair_stats(void* ws, long long* out, void* stream);

/* Static description of a status code. */
const char* digs_status_string(digs_status s);

#ifdef __cplusplus
}
#endif
#endif /* DIGS_H */
