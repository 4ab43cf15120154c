// Fused Adam over every parameter group of a reconstruction in one launch (Sec. 4.2: the reference
// Gaussians and the space / time B-spline grids are updated jointly by Adam).  Scales are optimised in
// log space and densities through a softplus, so both stay positive; the update is applied to the
// physical values directly.
#include "digs_internal.h"

namespace digs {

constexpr int kMaxAdamGroups = 8;

struct AdamParams {
  AdamGroup g[kMaxAdamGroups];
  int ng;
  long long total;
  float b1, b2, eps, bc1, bc2;
  const int* iter_dev;  // device step counter (0-based), or null: bc1, bc2 and the groups' lr apply
  int total_iters;
};

__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamParams P) {
  long long stride = (long long)gridDim.x * blockDim.x;
  float bc1 = P.bc1, bc2 = P.bc2, t = -1.f;
  if (P.iter_dev) {  // schedule of the step the device counter names
    const int it = *P.iter_dev;
    bc1 = 1.f - powf(P.b1, (float)(it + 1));
    bc2 = 1.f - powf(P.b2, (float)(it + 1));
    t = P.total_iters > 1 ? fminf(fmaxf((float)it / (float)(P.total_iters - 1), 0.f), 1.f) : 0.f;
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.total; i += stride) {
    int k = 0;
    while (k + 1 < P.ng && i >= P.g[k + 1].off) ++k;
    const AdamGroup& G = P.g[k];
    long long j = i - G.off;
    float p = G.p[j];
    float g = G.g[j];
    if (G.kind == 1) g *= p;                 // d/d(log s)
    else if (G.kind == 2) g *= -expm1f(-p);  // d/dtheta with rho = softplus(theta): sigmoid(theta) = 1 - e^-rho
    float m = fmaf(P.b1, G.m[j], (1.f - P.b1) * g);
    float v = fmaf(P.b2, G.v[j], (1.f - P.b2) * g * g);
    G.m[j] = m;
    G.v[j] = v;
    const float lr = t >= 0.f ? fmaf(G.lr_end - G.lr, t, G.lr) : G.lr;
    float step = lr * (m / bc1) / (sqrtf(v / bc2) + P.eps);
    if (G.kind == 1) p *= expf(-step);
    else if (G.kind == 2) p = log1pf(expm1f(p) * expf(-step));
    else p -= step;
    G.p[j] = p;
  }
}

__global__ void k_iter_bump(int* iter_dev) { *iter_dev += 1; }

cudaError_t launch_adam(const AdamGroup* groups, int ngroups, float beta1, float beta2, float eps, int step,
                        int* iter_dev, int total_iters, cudaStream_t st) {
  if (ngroups > kMaxAdamGroups) return cudaErrorInvalidValue;
  AdamParams P;
  P.ng = 0;
  long long off = 0;
  for (int i = 0; i < ngroups; ++i) {
    if (groups[i].n <= 0) continue;
    P.g[P.ng] = groups[i];
    P.g[P.ng].off = off;
    off += groups[i].n;
    ++P.ng;
  }
  P.total = off;
  if (off == 0) return cudaSuccess;
  P.b1 = beta1;
  P.b2 = beta2;
  P.eps = eps;
  P.bc1 = 1.f - powf(beta1, (float)step);
  P.bc2 = 1.f - powf(beta2, (float)step);
  P.iter_dev = iter_dev;
  P.total_iters = total_iters;
  long long blocks = (off + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_adam<<<(unsigned)blocks, 256, 0, st>>>(P);
  note_launches(1);
  if (iter_dev) {
    k_iter_bump<<<1, 1, 0, st>>>(iter_dev);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace digs
