// The largest dynamic shared memory a block may opt into, set once per
// kernel as its limit: a constant value, so host threads that launch the same
// kernel with different sizes never lower it under one another's launch.
#pragma once
#include <cuda_runtime.h>

inline int smem_optin_bytes() {
  static const int v = [] {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || b <= 0) {
      cudaGetLastError();
      b = 227 * 1024;
    }
    return b;
  }();
  return v;
}

template <class K> inline void smem_optin(K* kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_bytes());
}
