// The 6-D pose entry points (the appendix "Alternating search over rotations
// and translations"): volume poses, the translation search at a fixed
// rotation, and the alternation of Algorithm 1's rotation search with the
// translation search.
#include <math.h>
#include <stdio.h>
#include "internal.cuh"

using namespace matcha;

namespace matcha {
void set_error_text(const char *msg);
}

namespace {

bool shift_args_ok(int max_shift, int upsample) {
  return max_shift >= 0 && max_shift <= 64 && upsample >= 1 && upsample <= 64;
}

matcha_status unsupported(const char *msg) {
  set_error_text(msg);
  return MATCHA_ERR_UNSUPPORTED;
}

matcha_status cuda_fail(cudaError_t e, const char *where) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
  set_error_text(msg);
  return MATCHA_ERR_CUDA;
}

__global__ void k_or_flags(int B, const int *__restrict__ src, int *__restrict__ dst) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) dst[b] |= src[b];
}

struct Pose6dWs {
  void *align_ws;
  size_t align_bytes;
  float *shifted, *rotated;
  ShiftWs sw;
  int *tflags, *best_p;
};

size_t carve_pose6d(const Plan &p, int B, int tstride, int max_shift, int upsample, char *base,
                    Pose6dWs *w, matcha_plan plan) {
  size_t align_bytes = 0;
  matcha_workspace_size(plan, B, &align_bytes);
  const size_t vox = (size_t)p.N * p.N * p.N;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *r = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return r;
  };
  w->align_ws = take(align_bytes);
  w->align_bytes = align_bytes;
  w->shifted = reinterpret_cast<float *>(take(sizeof(float) * vox * B));
  w->rotated = reinterpret_cast<float *>(take(sizeof(float) * vox * B));
  w->tflags = reinterpret_cast<int *>(take(sizeof(int) * (size_t)B));
  w->best_p = reinterpret_cast<int *>(take(sizeof(int) * (size_t)B));
  size_t sbytes = shift_ws_bytes(p, B, max_shift, upsample, nullptr, nullptr);
  char *sb = take(sbytes);
  shift_ws_bytes(p, B, max_shift, upsample, sb, &w->sw);
  (void)tstride;
  return off;
}

}  // namespace

extern "C" matcha_status matcha_transform_volumes(int N, const float *vols, int B, int vol_stride,
                                                  const double *R, const double *shift,
                                                  int precision, float *out, void *stream) {
  if (N < 4 || N > 512 || B < 0 || (vol_stride != 0 && vol_stride != 1)) return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  if (!vols || !out) return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  if (precision < MATCHA_FP64 || precision > MATCHA_BF16) return MATCHA_ERR_INVALID_ARG;
  const long vox = (long)N * N * N;
  cudaError_t e = launch_pose_volumes(N, vols, B, vol_stride ? vox : 0, R, shift,
                                      precision == MATCHA_FP64, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "matcha_transform_volumes");
  return MATCHA_OK;
}

extern "C" matcha_status matcha_shift_search_workspace_size(matcha_plan plan, int B, int max_shift,
                                                            int upsample, size_t *bytes) {
  if (!plan || !bytes || B < 0 || !shift_args_ok(max_shift, upsample)) return MATCHA_ERR_INVALID_ARG;
  const Plan &p = *reinterpret_cast<const Plan *>(plan);
  *bytes = shift_ws_bytes(p, B, max_shift, upsample, nullptr, nullptr);
  return MATCHA_OK;
}

extern "C" matcha_status matcha_shift_search(matcha_plan plan, const float *particles,
                                             const float *rotated, int B, int max_shift,
                                             int upsample, const double *R, double *t,
                                             double *tau, double *cc, int *flags, void *ws,
                                             size_t ws_bytes, void *stream) {
  if (!plan || B < 0 || !shift_args_ok(max_shift, upsample)) return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  if (!particles || !rotated || !t || !cc || !flags || !ws || (tau && !R))
    return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return MATCHA_ERR_INVALID_ARG;
  const Plan &p = *reinterpret_cast<const Plan *>(plan);
  if (!p.fft_npass) return unsupported("matcha_shift_search: the box edge N must factor into 2, 3 and 5");
  if (2 * max_shift + 1 > p.N) return MATCHA_ERR_INVALID_ARG;
  ShiftWs w;
  size_t need = shift_ws_bytes(p, B, max_shift, upsample, (char *)ws, &w);
  if (ws_bytes < need) return MATCHA_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = p.fp64 ? launch_shift_search<double>(p, particles, rotated, B, max_shift, upsample,
                                                       R, w, t, tau, cc, flags, st)
                         : launch_shift_search<float>(p, particles, rotated, B, max_shift, upsample,
                                                      R, w, t, tau, cc, flags, st);
  if (e != cudaSuccess) return cuda_fail(e, "matcha_shift_search");
  return MATCHA_OK;
}

extern "C" matcha_status matcha_align6d_workspace_size(matcha_plan plan, int B, int tstride,
                                                       int max_shift, int upsample, size_t *bytes) {
  if (!plan || !bytes || B < 0 || (tstride != 0 && tstride != 1) || !shift_args_ok(max_shift, upsample))
    return MATCHA_ERR_INVALID_ARG;
  const Plan &p = *reinterpret_cast<const Plan *>(plan);
  Pose6dWs w;
  *bytes = carve_pose6d(p, B, tstride, max_shift, upsample, nullptr, &w, plan);
  return MATCHA_OK;
}

extern "C" matcha_status matcha_align6d(matcha_plan plan, const float *particles,
                                        const float *templates, int B, int tstride, int rounds,
                                        int max_shift, int upsample, double *euler, double *R,
                                        double *tau, double *t, double *score, double *cc,
                                        int *flags, void *ws, size_t ws_bytes, void *stream) {
  if (!plan || B < 0 || (tstride != 0 && tstride != 1) || rounds < 1 || rounds > 16 ||
      !shift_args_ok(max_shift, upsample))
    return MATCHA_ERR_INVALID_ARG;
  if (B == 0) return MATCHA_OK;
  if (!particles || !templates || !euler || !R || !tau || !t || !score || !cc || !flags || !ws)
    return MATCHA_ERR_INVALID_ARG;
  if (B > 65535) return MATCHA_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return MATCHA_ERR_INVALID_ARG;
  const Plan &p = *reinterpret_cast<const Plan *>(plan);
  if (!p.fft_npass) return unsupported("matcha_align6d: the box edge N must factor into 2, 3 and 5");
  if (2 * max_shift + 1 > p.N) return MATCHA_ERR_INVALID_ARG;
  Pose6dWs w;
  size_t need = carve_pose6d(p, B, tstride, max_shift, upsample, (char *)ws, &w, plan);
  if (ws_bytes < need) return MATCHA_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const long vox = (long)p.N * p.N * p.N;
  const bool fp64 = p.fp64;
  int *best_p = w.best_p;  // the rotation's best candidate is not an output here
  for (int r = 0; r < rounds; ++r) {
    // rotation search on (f, S_tau h): the template itself in the first round
    const float *tr = templates;
    int ts = tstride;
    if (r > 0) {
      cudaError_t e = launch_pose_volumes(p.N, templates, B, tstride ? vox : 0, nullptr, tau, fp64,
                                          w.shifted, st);
      if (e != cudaSuccess) return cuda_fail(e, "matcha_align6d: shift");
      tr = w.shifted;
      ts = 1;
    }
    matcha_status s = matcha_align(plan, particles, tr, B, ts, nullptr, euler, R, score, best_p,
                                   flags, w.align_ws, w.align_bytes, stream);
    if (s != MATCHA_OK) return s;
    // translation search of the rotated template u = g o h
    cudaError_t e = launch_pose_volumes(p.N, templates, B, tstride ? vox : 0, R, nullptr, fp64,
                                        w.rotated, st);
    if (e != cudaSuccess) return cuda_fail(e, "matcha_align6d: rotate");
    e = fp64 ? launch_shift_search<double>(p, particles, w.rotated, B, max_shift, upsample, R, w.sw,
                                           t, tau, cc, w.tflags, st)
             : launch_shift_search<float>(p, particles, w.rotated, B, max_shift, upsample, R, w.sw,
                                          t, tau, cc, w.tflags, st);
    if (e != cudaSuccess) return cuda_fail(e, "matcha_align6d: shift search");
  }
  k_or_flags<<<(B + 255) / 256, 256, 0, st>>>(B, w.tflags, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "matcha_align6d");
  return MATCHA_OK;
}
