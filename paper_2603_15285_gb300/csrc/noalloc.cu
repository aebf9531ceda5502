// matcha_soft_search_noalloc: the SOFFT grid search with its grid scratch in a
// fixed device array compiled into the library, for callers that must not
// allocate device memory themselves.
//
// Who needs it: a host application whose device memory is owned by one
// allocator (a framework's caching allocator, or a pool sized once at
// start-up) may forbid side allocations, and a latency-critical loop cannot
// afford cudaMalloc/cudaFree, which can synchronise the device.  Such a
// caller still owns the inputs (c) and the candidate outputs; only the
// grid scratch, which matcha_soft_search takes from the caller, moves into
// the library.
//
// The array below is a host-side stand-in in host code: host code must not
// pass &g_soft_grid_scratch to a kernel.  The device address is obtained once
// per device with cudaGetSymbolAddress, with that device current, during the
// first call on that device, and cached.  Every call on a device shares the
// one array; calls whose kernels overlap on the GPU (e.g. on two streams)
// race on it.  The grid kernel overwrites every grid value it later reads,
// so nothing in the array has to start at zero.
#include <mutex>
#include <stdio.h>
#include "internal.cuh"

namespace matcha {
void set_error_text(const char *msg);
}

namespace {

constexpr size_t kGridScratchBytes = size_t(MATCHA_NOALLOC_GRID_BYTES);
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_soft_grid_scratch[kGridScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_soft_grid_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" matcha_status matcha_soft_search_noalloc(matcha_plan plan, const void *c, int B,
                                                     const int *P_per, int *idx, double *euler,
                                                     double *score, int *n_cand, void *stream) {
  using namespace matcha;
  if (!plan || B < 0 || (B > 0 && (!c || !idx || !euler || !score || !n_cand)))
    return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  const Plan &p = *reinterpret_cast<const Plan *>(plan);
  size_t per = (size_t)p.ns * p.ns * p.ns * (p.fp64 ? 8 : 4);
  if ((size_t)B * per > kGridScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "matcha_soft_search_noalloc: B=%d needs %zu bytes of grid scratch, the built-in "
             "array holds %zu (at most %zu particles per call for this plan)",
             B, (size_t)B * per, kGridScratchBytes, kGridScratchBytes / per);
    set_error_text(msg);
    return MATCHA_ERR_UNSUPPORTED;
  }
  void *grid = nullptr;
  cudaError_t e = scratch_address(&grid);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "matcha_soft_search_noalloc: cudaGetSymbolAddress: %s",
             cudaGetErrorString(e));
    set_error_text(msg);
    return MATCHA_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  e = p.fp64 ? launch_soft<double>(p, (const double *)c, B, P_per, (double *)grid, idx, euler,
                                   score, n_cand, st)
             : launch_soft<float>(p, (const float *)c, B, P_per, (float *)grid, idx, euler, score,
                                  n_cand, st);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "matcha_soft_search_noalloc: %s", cudaGetErrorString(e));
    set_error_text(msg);
    return MATCHA_ERR_CUDA;
  }
  return MATCHA_OK;
}
