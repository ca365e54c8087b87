// Measured FP64 FMA rate of the current device: the roofline denominator of
// the library's FP64 kernels (mean and mixing length, shared-matrix assembly,
// right-hand sides, FP64 residuals), which on this architecture can be
// bound by the FP64 pipe rather than by memory.  The paper has no
// counterpart; this is a property of the hardware the library runs on.
#include <cstdint>

#include "kernels.h"

namespace {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_ITERS = 2048;

// FMA_CHAINS independent dependent chains per thread; the result is stored
// only if it is a value no input produces, so nothing is optimised away
__global__ void k_fp64_fma(double seed, double* sink) {
  double a[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) a[c] = seed + (double)(threadIdx.x + c);
  const double m = 0.999999999, q = 1e-9;
  for (int it = 0; it < FMA_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) a[c] = fma(a[c], m, q);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) s += a[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int mhde_fp64_fma_rate(void* stream, double* tflops) {
  if (!tflops) return MHDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MHDE_ECUDA;
  const int threads = 256, blocks = nsm * 8;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MHDE_ECUDA;
  k_fp64_fma<<<blocks, threads, 0, st>>>(1.0, nullptr);           // warm-up
  cudaEventRecord(e0, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) k_fp64_fma<<<blocks, threads, 0, st>>>(1.0 + r, nullptr);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                  cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || ms <= 0.f) return MHDE_ECUDA;
  const double flops = 2.0 * FMA_CHAINS * FMA_ITERS * (double)threads * blocks * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return MHDE_OK;
}
