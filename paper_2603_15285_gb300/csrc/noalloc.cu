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
// Only plans whose SOFFT grid is too large for the fused on-chip kernels (large
// L0, e.g. L0 = 30 with K = 2: 124^3 points per particle) write the grid to
// memory; for them the grid lives in the array below.  The other plans need no
// scratch at all: their fused kernels keep the grid on chip, so the call
// passes no grid and has no batch limit beyond matcha_soft_search's.
//
// The array's name is a host-side stand-in in host code: host code must not
// pass &g_soft_grid_scratch to a kernel.  The device address is looked up with
// cudaGetSymbolAddress, with the plan's device current, by the first call that
// needs it for a plan, and kept in that plan (a plan belongs to one device
// and one context, so the address cannot outlive it: after cudaDeviceReset
// both are gone and a new plan looks the address up again).  Every call on a
// device shares the one array; calls whose kernels overlap on the GPU (e.g.
// on two streams) race on it.  The grid kernel overwrites every grid value it
// later reads, so nothing in the array has to start at zero.
#include <mutex>
#include <stdio.h>
#include "internal.cuh"

namespace matcha {
void set_error_text(const char *msg);
}

namespace {

constexpr size_t kGridScratchBytes = size_t(MATCHA_NOALLOC_GRID_BYTES);

__device__ __align__(256) unsigned char g_soft_grid_scratch[kGridScratchBytes];

std::mutex g_scratch_mu;

// Device address of the scratch array for a plan (looked up once per plan,
// with the plan's device current).
cudaError_t scratch_address(matcha::Plan &p, void **out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!p.noalloc_grid) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != p.device) return cudaErrorInvalidDevice;
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_soft_grid_scratch);
    if (e != cudaSuccess) return e;
    p.noalloc_grid = ptr;
  }
  *out = p.noalloc_grid;
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
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  Plan &p = *reinterpret_cast<Plan *>(plan);
  void *grid = nullptr;  // the fused kernels keep the grid on chip and need none
  if (!soft_grid_optional(p)) {
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
    cudaError_t e = scratch_address(p, &grid);
    if (e != cudaSuccess) {
      char msg[256];
      snprintf(msg, sizeof(msg), "matcha_soft_search_noalloc: scratch address on device %d: %s",
               p.device, cudaGetErrorString(e));
      set_error_text(msg);
      return MATCHA_ERR_CUDA;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p.fp64 ? launch_soft<double>(p, (const double *)c, B, P_per, (double *)grid, idx,
                                               euler, score, n_cand, st)
                         : launch_soft<float>(p, (const float *)c, B, P_per, (float *)grid, idx,
                                              euler, score, n_cand, st);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "matcha_soft_search_noalloc: %s", cudaGetErrorString(e));
    set_error_text(msg);
    return MATCHA_ERR_CUDA;
  }
  return MATCHA_OK;
}
