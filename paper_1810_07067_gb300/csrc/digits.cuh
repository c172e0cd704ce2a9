// Exact digit slicing for FP64-accurate products on BF16 tensor cores: the
// operand tile layout of the MMAs and the fixed-point digits of a value.
#pragma once
#include <cuda_runtime.h>
#include <cstring>

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

// The same scale as its exponent E (scale = 2^E).
__device__ __forceinline__ int pow2_scale_exp(double mx) {
  if (!(mx > 0.0)) return 0;
  int e;
  frexp(mx, &e);
  return e + 1;
}

// The bits of |v| as an unsigned integer: for finite v their order is the
// order of |v|, so row maxima can be taken on the integer pipe.
__host__ __device__ __forceinline__ unsigned long long abs_bits(double v) {
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  memcpy(&b, &v, sizeof b);
#endif
  return b & 0x7FFFFFFFFFFFFFFFull;
}

// round(v 2^S), ties to even, from the sign, exponent and significand of v
// in integer arithmetic (on the sampling kernels the FP64 pipe is the
// scarce unit): for |v 2^S| < 2^55 the value of __double2ll_rn(v * 2^S)
// wherever that product is exact, and exact where it is not.
__host__ __device__ __forceinline__ long long fixed_rn(double v, int S) {
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  memcpy(&b, &v, sizeof b);
#endif
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  int e = 1;  // subnormals: significand without the leading one, exponent of the smallest normal
  if (ex) { mant |= 1ull << 52; e = ex; }
  const int sh = e - 1075 + S;  // v 2^S = mant 2^sh
  unsigned long long q;
  if (sh >= 0) {
    q = sh < 63 ? mant << sh : 0ull;  // sh >= 63 only for inf and NaN
  } else if (sh < -54) {
    q = 0ull;                          // mant 2^sh < 1/2
  } else {
    const int r = -sh;
    q = mant >> r;
    const unsigned long long rem = mant - (q << r), half = 1ull << (r - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

// Digits of a value v in (-1/2, 1/2) held as the fixed-point integer
// F = round(v 2^56), written in balanced base 128 from the least significant
// digit up, on two 28-bit halves in 32-bit integer arithmetic:
// d = ((F + 64) mod 128) - 64, F <- (F - d) / 128; the low half's carry joins
// the high half, and the top digit ends in [-64, 64].  v = sum_s d_s 2^{-7(s+1)}
// up to the rounding of F.
__host__ __device__ __forceinline__ void digits28(long long F, int* d) {
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

