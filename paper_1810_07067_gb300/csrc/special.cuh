// Stable entire functions of u = rho^2 used by the split modal kernels, and
// the Laplace-type modal coefficients P_m, S_m (Section 4, eqs. lm, pm;
// appendix recurrences).
//
// For x = k sqrt(u) (complex k allowed):
//   sinc(x) = sin x / x                     (= j0)
//   sig1(x) = (x cos x - sin x) / x^3       (= -j1(x)/x, = sinc'(x)/x)
//   sig2(x) = ((3-x^2) sin x - 3x cos x)/x^5 (= j2(x)/x^2, = sig1'(x)/x)
//   phi2(x) = (1 + sinc(x/2)^2 - 2 sinc x) / (4 x^2)
//   phi3(x) = (sinc(x/2) sig1(x/2)/2 - 2 sig1(x)) / 8
// all even entire functions of x, hence entire in u.  Taylor series are used
// for |x| < 2 and the closed forms above otherwise.
#pragma once
#include "cplx.cuh"

#define SPECIAL_NTERM 18

struct SeriesTables {
  double sinc[SPECIAL_NTERM];  // coefficient of (x^2)^n
  double sig1[SPECIAL_NTERM];
  double sig2[SPECIAL_NTERM];
  double phi2[SPECIAL_NTERM];
  double phi3[SPECIAL_NTERM];
  double hsinc[SPECIAL_NTERM];  // sinc[p] / 4^p: sinc at x/2 as a series in x^2
  double hsig1[SPECIAL_NTERM];  // sig1[p] / 4^p
};

// Fill the series tables on the host (exact rationals evaluated in double).
inline void fill_series_tables(SeriesTables* t) {
  // c_n = (-1)^n / (2n+1)!  ;  sinc = sum c_n x^(2n)
  // sig1 = sum_{n>=1} 2n c_n x^(2n-2)
  // sig2 = sum_{n>=2} 2n (2n-2) c_n x^(2n-4)
  // phi2 = sum_{n>=2} (-1)^n (n-1/2) x^(2n-4) / (2n)!
  // phi3 = sum_{n>=2} (-1)^n (n-1/2)(n-1) x^(2n-4) / (2n)!
  double fact[2 * SPECIAL_NTERM + 8];
  fact[0] = 1.0;
  for (int i = 1; i < 2 * SPECIAL_NTERM + 8; ++i) fact[i] = fact[i - 1] * i;
  for (int p = 0; p < SPECIAL_NTERM; ++p) {
    double sg = (p % 2) ? -1.0 : 1.0;
    t->sinc[p] = sg / fact[2 * p + 1];
    int n1 = p + 1;  // sig1 power p <- n = p+1
    t->sig1[p] = 2.0 * n1 * ((n1 % 2) ? -1.0 : 1.0) / fact[2 * n1 + 1];
    int n2 = p + 2;  // sig2, phi2, phi3 power p <- n = p+2
    double sg2 = (n2 % 2) ? -1.0 : 1.0;
    t->sig2[p] = 2.0 * n2 * (2.0 * n2 - 2.0) * sg2 / fact[2 * n2 + 1];
    t->phi2[p] = sg2 * (n2 - 0.5) / fact[2 * n2];
    t->phi3[p] = sg2 * (n2 - 0.5) * (n2 - 1.0) / fact[2 * n2];
    t->hsinc[p] = std::ldexp(t->sinc[p], -2 * p);  // exact: a power of two
    t->hsig1[p] = std::ldexp(t->sig1[p], -2 * p);
  }
}

// terms needed for |x^2| <= a2 so that the truncated tail is below 1e-17
// relative (the coefficients decay at least like 4^n / (2n)!)
HD int series_terms(double a2) {
  return a2 < 0.0625 ? 7 : (a2 < 0.25 ? 8 : (a2 < 1.0 ? 10 : (a2 < 2.25 ? 12 : (a2 < 4.0 ? 14 : SPECIAL_NTERM))));
}

HD cd horner(const double* c, cd x2, int nt = SPECIAL_NTERM) {
  cd acc = C(c[nt - 1]);
  for (int p = nt - 2; p >= 0; --p) acc = fma(acc, x2, C(c[p]));
  return acc;
}

struct SphFun {
  cd sinc, sig1, sig2;
};

// sinc, sig1, sig2 at x; s, c are sin x, cos x (used only when |x| >= 2)
HD SphFun sph_closed(cd x, cd s, cd c) {
  cd xi = C(1.0) / x;
  cd xi2 = xi * xi;
  SphFun f;
  f.sinc = s * xi;
  f.sig1 = (x * c - s) * xi2 * xi;
  f.sig2 = ((C(3.0) - x * x) * s - 3.0 * (x * c)) * xi2 * xi2 * xi;
  return f;
}

HD SphFun sph_series(const SeriesTables& T, cd x2, bool need_sig2 = true) {
  int nt = series_terms(norm2(x2) > 0 ? sqrt(norm2(x2)) : 0.0);
  SphFun f;
  f.sinc = horner(T.sinc, x2, nt);
  f.sig1 = horner(T.sig1, x2, nt);
  f.sig2 = need_sig2 ? horner(T.sig2, x2, nt) : C(0.0);
  return f;
}

// Per-wavenumber entire functions at sqrt(u) = su.
struct Ent {
  cd C;     // cos x
  cd S;     // sin x / sqrt(u) = k sinc x
  cd Gam;   // C'(u) - (C(u)-1)/(2u)
  cd Gam2;  // (Gam(u) - Gam(0)) / u
  cd Gamp;  // Gam'(u)
  cd Sp;    // S'(u)
  cd Spp;   // S''(u)
};

struct KPow {
  cd k, k2, k3, k4, k5;
};

HD KPow kpow(cd k) {
  KPow p;
  p.k = k; p.k2 = k * k; p.k3 = p.k2 * k; p.k4 = p.k2 * p.k2; p.k5 = p.k4 * k;
  return p;
}

HD Ent entire(const SeriesTables& T, const KPow& kp, double su) {
  cd x = kp.k * su;
  cd h = 0.5 * x;
  cd x2 = x * x;
  double ax = cabs(x);
  SphFun fx, fh;
  cd cosx;
  cd phi2, phi3;
  if (ax < 2.0) {
    // the seven series in x^2 share one table of powers: per term one complex
    // product for the power and a real-times-complex update per series
    // (half-argument series from the coefficients scaled by 4^-p)
    const int nt = series_terms(ax * ax);
    cd P = C(1.0), s0 = C(0.0), s1 = C(0.0), s2 = C(0.0), h0 = C(0.0), h1 = C(0.0), p2 = C(0.0), p3 = C(0.0);
    for (int p = 0; p < nt; ++p) {
      s0 = fma(T.sinc[p], P, s0); s1 = fma(T.sig1[p], P, s1); s2 = fma(T.sig2[p], P, s2);
      h0 = fma(T.hsinc[p], P, h0); h1 = fma(T.hsig1[p], P, h1);
      p2 = fma(T.phi2[p], P, p2); p3 = fma(T.phi3[p], P, p3);
      P = P * x2;
    }
    fx.sinc = s0; fx.sig1 = s1; fx.sig2 = s2;
    fh.sinc = h0; fh.sig1 = h1; fh.sig2 = C(0.0);
    phi2 = p2; phi3 = p3;
  } else {
    cd sh, chh;
    csincos(h, &sh, &chh);
    cd sx = 2.0 * (sh * chh);
    cd cx = C(1.0) - 2.0 * (sh * sh);
    fx = sph_closed(x, sx, cx);
    if (ax < 4.0) fh = sph_series(T, 0.25 * x2, false);
    else fh = sph_closed(h, sh, chh);
  }
  // cos x = 1 - 2 sin^2(x/2) = 1 - (x^2/2) sinc(x/2)^2  (stable for all x)
  cosx = C(1.0) - 0.5 * (x2 * (fh.sinc * fh.sinc));
  if (ax >= 2.0) {
    phi2 = (C(1.0) + fh.sinc * fh.sinc - 2.0 * fx.sinc) / (4.0 * x2);
    phi3 = (0.5 * (fh.sinc * fh.sig1) - 2.0 * fx.sig1) * 0.125;
  }
  Ent e;
  e.C = cosx;
  e.S = kp.k * fx.sinc;
  e.Gam = -0.5 * (kp.k2 * fx.sinc) + 0.25 * (kp.k2 * (fh.sinc * fh.sinc));
  e.Gam2 = kp.k4 * phi2;
  e.Gamp = kp.k4 * phi3;
  e.Sp = 0.5 * (kp.k3 * fx.sig1);
  e.Spp = 0.25 * (kp.k5 * fx.sig2);
  return e;
}

// Real-argument versions (real wavenumber): same functions, real arithmetic.
HD double horner_r(const double* c, double x2, int nt) {
  double acc = c[nt - 1];
  for (int p = nt - 2; p >= 0; --p) acc = fma(acc, x2, c[p]);
  return acc;
}

HD Ent entire_real(const SeriesTables& T, double k, double su) {
  const double x = k * su, h = 0.5 * x, x2 = x * x, ax = fabs(x);
  double sx_c, s1x, s2x, sh_c, s1h, cosx, phi2, phi3;
  if (ax < 2.0) {
    int nt = series_terms(x2);
    sx_c = horner_r(T.sinc, x2, nt);
    s1x = horner_r(T.sig1, x2, nt);
    s2x = horner_r(T.sig2, x2, nt);
    int nh = series_terms(0.25 * x2);
    sh_c = horner_r(T.sinc, 0.25 * x2, nh);
    s1h = horner_r(T.sig1, 0.25 * x2, nh);
    phi2 = horner_r(T.phi2, x2, nt);
    phi3 = horner_r(T.phi3, x2, nt);
  } else {
    double sh, chh;
#ifdef __CUDA_ARCH__
    sincos(h, &sh, &chh);
#else
    sh = std::sin(h); chh = std::cos(h);
#endif
    const double sx = 2.0 * sh * chh, cx = 1.0 - 2.0 * sh * sh;
    const double xi = 1.0 / x, xi2 = xi * xi;
    sx_c = sx * xi;
    s1x = (x * cx - sx) * xi2 * xi;
    s2x = ((3.0 - x2) * sx - 3.0 * x * cx) * xi2 * xi2 * xi;
    if (ax < 4.0) {
      int nh = series_terms(0.25 * x2);
      sh_c = horner_r(T.sinc, 0.25 * x2, nh);
      s1h = horner_r(T.sig1, 0.25 * x2, nh);
    } else {
      const double hi = 1.0 / h;
      sh_c = sh * hi;
      s1h = (h * chh - sh) * hi * hi * hi;
    }
    phi2 = (1.0 + sh_c * sh_c - 2.0 * sx_c) / (4.0 * x2);
    phi3 = (0.5 * sh_c * s1h - 2.0 * s1x) * 0.125;
  }
  cosx = 1.0 - 0.5 * x2 * sh_c * sh_c;
  const double k2 = k * k, k3 = k2 * k, k4 = k2 * k2, k5 = k4 * k;
  Ent e;
  e.C = C(cosx);
  e.S = C(k * sx_c);
  e.Gam = C(-0.5 * k2 * sx_c + 0.25 * k2 * sh_c * sh_c);
  e.Gam2 = C(k4 * phi2);
  e.Gamp = C(k4 * phi3);
  e.Sp = C(0.5 * k3 * s1x);
  e.Spp = C(0.25 * k5 * s2x);
  return e;
}

// Complete elliptic integral of the first kind from the complementary modulus
// kp = sqrt(1 - kappa^2): K = pi / (2 AGM(1, kp)).
HD double ellipk_c(double kp) {
  double a = 1.0, b = kp;
  for (int it = 0; it < 64; ++it) {
    double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
    if (fabs(a - b) <= 1e-16 * a) break;
  }
  return M_PI / (a + b);
}

// Carlson's symmetric integral R_D(x, y, z) by the duplication theorem with
// the fifth-order series of DLMF 19.36.2 (x, y >= 0, z > 0).
HD double carlson_rd(double x, double y, double z) {
  double sum = 0.0, fac = 1.0, A = 0.0, X = 0.0, Y = 0.0;
  for (int it = 0; it < 200; ++it) {
    double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
    double lam = sx * sy + sx * sz + sy * sz;
    sum += fac / (sz * (z + lam));
    fac *= 0.25;
    x = 0.25 * (x + lam); y = 0.25 * (y + lam); z = 0.25 * (z + lam);
    A = (x + y + 3.0 * z) * 0.2;
    X = 1.0 - x / A; Y = 1.0 - y / A;
    double Zt = 1.0 - z / A;
    if (fmax(fabs(X), fmax(fabs(Y), fabs(Zt))) < 1e-3) break;
  }
  double Z = -(X + Y) / 3.0, XY = X * Y, Z2 = Z * Z;
  double E2 = XY - 6.0 * Z2, E3 = (3.0 * XY - 8.0 * Z2) * Z, E4 = 3.0 * (XY - Z2) * Z2, E5 = XY * Z2 * Z;
  double ser = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0 - 9.0 * E2 * E3 / 52.0 +
               3.0 * E5 / 26.0;
  return 3.0 * sum + fac * ser / (A * sqrt(A));
}

// Complete elliptic integral of the second kind without cancellation near
// kappa -> 1: E = (kp^2/3) [R_D(0, kp^2, 1) + R_D(0, 1, kp^2)] (DLMF 19.25.1).
HD double ellipe_c(double kp2) { return kp2 * (carlson_rd(0.0, kp2, 1.0) + carlson_rd(0.0, 1.0, kp2)) / 3.0; }
