// FP32 throughput probe: the measured denominator of the ALU rooflines.
//
// Not part of the alignment path.  Every thread runs independent FMA chains
// (paired FP32x2 FMAs with variant 1, scalar FMAs with variant 0) on values
// that stay bounded (x <- 0.999 x + 1e-7), long enough that launch overhead
// is negligible; the caller times the launch with CUDA events on its stream
// and divides the flops (2 per FMA lane) by the elapsed time.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;

__global__ void k_ffma2_peak(float *out, long iters) {
  float2 acc[CHAINS];
  const float2 a = make_float2(0.999f, 0.999f), c = make_float2(1e-7f, 1e-7f);
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) acc[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
  for (long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc[k] = __ffma2_rn(acc[k], a, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += acc[k].x + acc[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma_peak(float *out, long iters) {
  float acc[2 * CHAINS];
#pragma unroll
  for (int k = 0; k < 2 * CHAINS; ++k) acc[k] = threadIdx.x * 1e-3f + k;
  for (long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 2 * CHAINS; ++k) acc[k] = fmaf(acc[k], 0.999f, 1e-7f);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * CHAINS; ++k) s += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Launches the probe: blocks x threads threads, `iters` trips of 16 FMA lanes
// per thread (flops = blocks * threads * iters * 32).  out: blocks * threads
// floats of device memory.  Returns the cudaError_t of the launch.
extern "C" int peak_fp32_launch(int variant, int blocks, int threads, long iters, float *out,
                                void *stream) {
  if (blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0 || !out)
    return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  if (variant == 1) k_ffma2_peak<<<blocks, threads, 0, st>>>(out, iters);
  else k_ffma_peak<<<blocks, threads, 0, st>>>(out, iters);
  return (int)cudaGetLastError();
}
