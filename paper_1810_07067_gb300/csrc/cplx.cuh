// Minimal complex128 arithmetic for host and device code.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define HD __host__ __device__ __forceinline__
#else
#define HD inline
#endif

struct cd {
  double x, y;
};

HD cd C(double a, double b = 0.0) { return cd{a, b}; }
HD cd operator+(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
HD cd operator-(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
HD cd operator-(cd a) { return cd{-a.x, -a.y}; }
HD cd operator*(cd a, cd b) { return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
HD cd operator*(double s, cd a) { return cd{s * a.x, s * a.y}; }
HD cd operator*(cd a, double s) { return cd{s * a.x, s * a.y}; }
HD cd operator/(cd a, double s) { return cd{a.x / s, a.y / s}; }
HD cd& operator+=(cd& a, cd b) { a.x += b.x; a.y += b.y; return a; }
HD cd& operator-=(cd& a, cd b) { a.x -= b.x; a.y -= b.y; return a; }
HD cd conj(cd a) { return cd{a.x, -a.y}; }
HD double norm2(cd a) { return a.x * a.x + a.y * a.y; }
HD double cabs(cd a) { return hypot(a.x, a.y); }
HD cd mul_i(cd a) { return cd{-a.y, a.x}; }  // i * a
HD cd operator/(cd a, cd b) {
  // scaled division (Smith's method)
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return cd{(a.x + a.y * r) / den, (a.y - a.x * r) / den};
  } else {
    double r = b.x / b.y, den = b.x * r + b.y;
    return cd{(a.x * r + a.y) / den, (a.y * r - a.x) / den};
  }
}
HD cd fma(cd a, cd b, cd c) {  // a*b + c
  return cd{fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
HD cd fma(double s, cd b, cd c) { return cd{fma(s, b.x, c.x), fma(s, b.y, c.y)}; }

// sin and cos of a complex argument x = a + ib
HD void csincos(cd z, cd* s, cd* c) {
  double sa, ca;
#ifdef __CUDA_ARCH__
  sincos(z.x, &sa, &ca);
#else
  sa = std::sin(z.x); ca = std::cos(z.x);
#endif
  double em = expm1(z.y), emn = expm1(-z.y);
  double ch = 1.0 + 0.5 * (em + emn), sh = 0.5 * (em - emn);
  *s = cd{sa * ch, ca * sh};
  *c = cd{ca * ch, -sa * sh};
}
// exp(i z)
HD cd cexpi(cd z) {
  double sa, ca;
#ifdef __CUDA_ARCH__
  sincos(z.x, &sa, &ca);
#else
  sa = std::sin(z.x); ca = std::cos(z.x);
#endif
  double e = exp(-z.y);
  return cd{e * ca, e * sa};
}
HD cd csqrt_principal(cd z) {
  double r = cabs(z);
  double re = sqrt(0.5 * (r + z.x));
  double im = sqrt(0.5 * fmax(r - z.x, 0.0));
  if (z.y < 0) im = -im;
  return cd{re, im};
}

// complex64 for the mixed-precision factors
struct cf {
  float x, y;
};
HD cf CF(float a, float b = 0.f) { return cf{a, b}; }
HD cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
HD cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
HD cf operator-(cf a) { return cf{-a.x, -a.y}; }
HD cf operator*(cf a, cf b) { return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
HD cf operator*(float s, cf a) { return cf{s * a.x, s * a.y}; }
HD cf& operator+=(cf& a, cf b) { a.x += b.x; a.y += b.y; return a; }
HD double norm2(cf a) { return (double)a.x * a.x + (double)a.y * a.y; }
// Smith's scaled division in FP32: the complex64 kernels divide once per
// column or step in every thread, and FP64 arithmetic is a small share of
// this part's issue rate.
HD cf operator/(cf a, cf b) {
  if (fabsf(b.x) >= fabsf(b.y)) {
    const float r = b.y / b.x, den = b.x + b.y * r;
    return cf{(a.x + a.y * r) / den, (a.y - a.x * r) / den};
  } else {
    const float r = b.x / b.y, den = b.x * r + b.y;
    return cf{(a.x * r + a.y) / den, (a.y * r - a.x) / den};
  }
}
HD cf fma(cf a, cf b, cf c) {
  return cf{fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y))};
}
template <class T> HD T czero();
template <> HD cd czero<cd>() { return cd{0.0, 0.0}; }
template <> HD cf czero<cf>() { return cf{0.f, 0.f}; }
template <class T> HD T cone();
template <> HD cd cone<cd>() { return cd{1.0, 0.0}; }
template <> HD cf cone<cf>() { return cf{1.f, 0.f}; }
HD cf to_cf(cd a) { return cf{(float)a.x, (float)a.y}; }
HD cd to_cd(cf a) { return cd{a.x, a.y}; }
