// digs_project_fwd_static: the forward projection with its scratch in a fixed, file-scope device array
// instead of a caller-provided workspace, for callers that cannot allocate device memory themselves.
//
// The array is DIGS_STATIC_SCRATCH_BYTES (32 MiB).  Every GPU on which the library's code is loaded
// holds it until the process exits.  All calls share it: a call overwrites what the previous one left,
// and two calls whose work overlaps on the GPU (different streams, or different host threads) race on it.
// Each call is synchronous (it waits for its stream to read the device status), so it is refused on a
// stream that is being captured.
#include <mutex>

#include "digs_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = DIGS_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on each device, looked up once per device.  In host code the
// symbol name only stands in for the array; the kernels must be given this address.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

digs_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DIGS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return DIGS_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return DIGS_OK;
}

}  // namespace

extern "C" digs_status digs_project_fwd_static(const DigsGaussians* g, const DigsLattice* lat, const float* phi,
                                               const float* w, const DigsView* views, int P, const DigsOpts* opts,
                                               float* proj, void* stream) {
  if (!g || !lat || !views || P < 0 || P > DIGS_MAX_VIEWS) return DIGS_ERR_ARG;
  void* base = nullptr;
  digs_status s = scratch_for_current_device(&base);
  if (s != DIGS_OK) return s;
  // Reject problems whose pair-independent scratch alone does not fit the array.
  int nu = P > 0 ? views[0].nu : 1, nv = P > 0 ? views[0].nv : 1;
  size_t fixed = digs_workspace_size(g->n, P, nu, nv, lat->R, 0, opts);
  if (fixed == 0 || fixed > kStaticScratchBytes) return DIGS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // The call ends by reading the device status back to the host, which a capturing stream cannot do.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return DIGS_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return DIGS_ERR_ARG;
  // The status block (error word, pair counts) must start at zero; the array keeps the last call's bytes.
  if (cudaMemsetAsync(base, 0, 256, st) != cudaSuccess) return DIGS_ERR_CUDA;
  s = digs_project_fwd(g, lat, phi, w, views, P, opts, proj, base, kStaticScratchBytes, stream);
  if (s != DIGS_OK) return s;
  // Wait for the call and report what the device recorded (DIGS_ERR_CAPACITY if the pairs did not fit).
  int h = 0;
  if (cudaMemcpyAsync(&h, base, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DIGS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DIGS_ERR_CUDA;
  return (digs_status)h;
}
