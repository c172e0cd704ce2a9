// Exact digit slicing for FP64-accurate products on BF16 tensor cores: the
// operand tile layout of the MMAs and the fixed-point digits of a value.
#pragma once
#include <cuda_runtime.h>

#ifndef OZ_S
#define OZ_S 8        // digits per value (7 bits each)
#endif

// offset of element (row r, k) inside a slice tile with R rows and 16 columns
// (core matrices of 8 x 8, row-group major; two core matrices along k)
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ double pow2_scale(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);               // mx = f 2^e, f in [1/2, 1)
  return ldexp(1.0, e + 1);    // |a| / scale < 1/2
}

// Digits of a value v in (-1/2, 1/2) held as the fixed-point integer
// F = round(v 2^56), written in balanced base 128 from the least significant
// digit up, on two 28-bit halves in 32-bit integer arithmetic:
// d = ((F + 64) mod 128) - 64, F <- (F - d) / 128; the low half's carry joins
// the high half, and the top digit ends in [-64, 64].  v = sum_s d_s 2^{-7(s+1)}
// up to the rounding of F.
__device__ __forceinline__ void digits28(long long F, int* d) {
  int lo = (int)(F & 0xFFFFFFFll), hi = (int)(F >> 28);
#pragma unroll
  for (int s = OZ_S - 1; s >= OZ_S / 2; --s) {
    const int dd = ((lo + 64) & 127) - 64;
    d[s] = dd;
    lo = (lo - dd) >> 7;
  }
  hi += lo;  // carry of the low half (0 or 1)
#pragma unroll
  for (int s = OZ_S / 2 - 1; s >= 1; --s) {
    const int dd = ((hi + 64) & 127) - 64;
    d[s] = dd;
    hi = (hi - dd) >> 7;
  }
  d[0] = hi;
}

