// Measurement support: the FP64 fused multiply-add rate of the device, the denominator of the sweep
// kernels' roofline (they are bound by FP64 issue, not by memory).  The paper has no counterpart.
//
// Every thread runs eight independent FMA chains (enough to cover the FP64 pipe's latency), on
// every SM, for a fixed number of iterations; the rate is the FMAs executed over the CUDA-event
// time of the launch.
#include <cuda_runtime.h>

#include "../../include/grape_hg.h"

namespace {

__global__ void __launch_bounds__(512) k_fma_rate(double* sink, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-9, x2 = x0 + 2e-9, x3 = x0 + 3e-9;
  double x4 = x0 + 4e-9, x5 = x0 + 5e-9, x6 = x0 + 6e-9, x7 = x0 + 7e-9;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  const double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == 0.125) sink[blockIdx.x] = s;   // never true for these inputs; keeps the chains alive
}

}  // namespace

extern "C" grape_status grape_fp64_fma_rate(int32_t device, double* gflops) {
  if (!gflops) return GRAPE_EINVAL;
  *gflops = 0.0;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return GRAPE_ECUDA;
  grape_status st = GRAPE_OK;
  int nsm = 0;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int threads = 512, iters = 20000;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&sink, (size_t)nsm * 2 * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = GRAPE_ECUDA;
  } else {
    const int blocks = 2 * nsm;
    k_fma_rate<<<blocks, threads>>>(sink, 200, 0.999999, 1e-7);   // warm-up (clocks, module load)
    cudaEventRecord(e0);
    k_fma_rate<<<blocks, threads>>>(sink, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
      st = GRAPE_ECUDA;
    else
      *gflops = 2.0 * 8.0 * (double)iters * blocks * threads / ((double)ms * 1e6);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  return st;
}
