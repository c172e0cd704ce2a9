// Peak FP64 arithmetic rate of the current device, measured by a register
// loop of fused multiply-adds (the denominator of the FP64 roofline of the
// kernel-evaluation and assembly stages, which run on the FP64 pipe).
#include <cuda_runtime.h>
#include <algorithm>
#include "mueller.h"

#define PROBE_CHAINS 8

// Every thread runs PROBE_CHAINS independent dependency chains of
// x <- x * a + b for `iters` steps: 2 flops per step and chain.  The values
// stay bounded (|a| < 1) and the sum is stored only under a condition that
// never holds, so that the loop is not removed.
__global__ void __launch_bounds__(256) dfma_probe_kernel(int iters, double a, double b, double* sink) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == -1.0) sink[0] = s;
}

extern "C" int mueller_fp64_peak(double* tflops, void* stream) {
  if (!tflops) return MUELLER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MUELLER_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 1 << 16;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_probe_kernel<<<blocks, threads, 0, s>>>(iters / 16, 0.999999, 1e-7, nullptr);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0, s);
    dfma_probe_kernel<<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, nullptr);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0); cudaEventDestroy(e1);
      return MUELLER_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return MUELLER_ECUDA;
  const double flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return MUELLER_OK;
}
