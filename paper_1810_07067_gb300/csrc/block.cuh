// The Mueller 4 x 4 block of one (target, source or column, mode) from the
// modal kernel spectra (Lemma 1 and the modal N and K operators, Section 3),
// for the GPU kernels and, host-callable, for host-side checks.
#pragma once
#include "cplx.cuh"
#include "green.cuh"

// Mueller 4x4 block for one (target, source-or-column, mode m >= 0) from an
// accessor R(sigma, f, mm): sigma 0 = r r' weight, 1 = r weight, 2 = r z' weight.
struct V2 { cd a, b; };  // coefficients of J^1, J^2
__host__ __device__ __forceinline__ V2 v2(cd a, cd b) { V2 v; v.a = a; v.b = b; return v; }
__host__ __device__ __forceinline__ V2 operator+(V2 x, V2 y) { return v2(x.a + y.a, x.b + y.b); }
__host__ __device__ __forceinline__ V2 operator-(V2 x, V2 y) { return v2(x.a - y.a, x.b - y.b); }
__host__ __device__ __forceinline__ V2 operator*(cd s, V2 x) { return v2(s * x.a, s * x.b); }
__host__ __device__ __forceinline__ V2 operator*(double s, V2 x) { return v2(s * x.a, s * x.b); }
__host__ __device__ __forceinline__ V2 operator-(V2 x) { return v2(-x.a, -x.b); }
// (i y) x for real y: two multiplies per complex entry instead of a complex product
__host__ __device__ __forceinline__ cd iy(double y, cd a) { return cd{-y * a.y, y * a.x}; }
__host__ __device__ __forceinline__ V2 iy(double y, V2 x) { return v2(iy(y, x.a), iy(y, x.b)); }

// The block from the gathered coefficients c1, c2 (of J^1 and J^2) and c3
// (of J^1 alone) of the nine families.  SIMPLE: k0^2 and k1^2 real, the
// coupling coefficients cEM and cHJ purely imaginary and the K factors
// aEJ = 1, aHM = -1 (real wavenumbers and eps0 = mu0 = 1, as AsmParams::simple
// records): the same block without the products by zero parts.
template <bool SIMPLE = false>
__host__ __device__ __forceinline__ void mueller_block_core(const V2* c1, const V2* c2, const cd* c3, int m,
                                                            const AsmParams& ap, double rt, double irt,
                                                            double rpt, double zpt, cd out[4][4]);

template <class Get>
__device__ void mueller_block(const Get& R, int m, const AsmParams& ap, double rt, double rpt, double zpt,
                              cd out[4][4]) {
  int a0 = m, ap1 = m + 1, am1 = (m >= 1) ? m - 1 : 1;
  V2 c1[NFAM], c2[NFAM];
  cd c3[NFAM];
#pragma unroll
  for (int f = 0; f < NFAM; ++f) {
    cd A0p = R(0, f, ap1), A0m = R(0, f, am1);
    cd A1p = R(1, f, ap1), A1m = R(1, f, am1);
    cd G2a = 0.5 * (A0p + A0m), G3a = 0.5 * (A0m - A0p);
    cd G2b = 0.5 * (A1p + A1m), G3b = 0.5 * (A1m - A1p);
    c1[f] = v2(G2a, -mul_i(G3b));
    c2[f] = v2(mul_i(G3a), G2b);
    c3[f] = R(2, f, a0);
  }
  mueller_block_core(c1, c2, c3, m, ap, rt, 1.0 / rt, rpt, zpt, out);
}

// The same block from one pair's unscaled spectra S[f * stride + (mode - base)]
// and its three quadrature weights fac (sigma = 0, 1, 2): the weights multiply
// the sums and differences of modes m +- 1 once instead of every term.  The
// block is linear in the spectra, so a common factor of the block (the L2
// row/column weight ratio) can ride in fac; irt = 1 / rt.
template <bool SIMPLE = false>
__host__ __device__ __forceinline__ void mueller_block_spec(const cd* S, int stride, int base, const double fac[3],
                                                            int m, const AsmParams& ap, double rt, double irt,
                                                            double rpt, double zpt, cd out[4][4]) {
  const int ap1 = m + 1 - base, am1 = ((m >= 1) ? m - 1 : 1) - base, a0 = m - base;
  const double h0 = 0.5 * fac[0], h1 = 0.5 * fac[1];
  V2 c1[NFAM], c2[NFAM];
  cd c3[NFAM];
#pragma unroll
  for (int f = 0; f < NFAM; ++f) {
    const cd sp = S[f * stride + ap1], sm = S[f * stride + am1];
    const cd sum = sp + sm, dif = sm - sp;
    c1[f] = v2(h0 * sum, -mul_i(h1 * dif));
    c2[f] = v2(mul_i(h0 * dif), h1 * sum);
    c3[f] = fac[2] * S[f * stride + a0];
  }
  mueller_block_core<SIMPLE>(c1, c2, c3, m, ap, rt, irt, rpt, zpt, out);
}

// k x for k = k0^2 or k1^2: a real scalar when SIMPLE
template <bool SIMPLE>
__host__ __device__ __forceinline__ V2 ksq_mul(cd k, V2 x) { return SIMPLE ? k.x * x : k * x; }
template <bool SIMPLE>
__host__ __device__ __forceinline__ cd ksq_mul(cd k, cd x) { return SIMPLE ? k.x * x : k * x; }
// c x for a coupling coefficient c: i Im(c) when SIMPLE
template <bool SIMPLE>
__host__ __device__ __forceinline__ V2 coup_mul(cd c, V2 x) { return SIMPLE ? iy(c.y, x) : c * x; }

template <bool SIMPLE>
__host__ __device__ __forceinline__ void mueller_block_core(const V2* c1, const V2* c2, const cd* c3, int m,
                                                            const AsmParams& ap, double rt, double irt,
                                                            double rpt, double zpt, cd out[4][4]) {
  const double irt2 = irt * irt;
  const double mr = m * irt, mr2 = m * irt2;  // i m / r_t and i m / r_t^2 act as iy(mr, .), iy(mr2, .)
  V2 Nt[2], Nth[2];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    int g = kk, dr = 2 + 2 * kk, dz = 3 + 2 * kk;
    Nt[kk] = v2(c1[dz].a - c3[dr], c1[dz].b);
    V2 t1 = c2[g] + rt * c2[dr] - iy((double)m, c1[g]);
    V2 t2 = v2(iy(mr, c3[g]) - c2[dz].a, -c2[dz].b);
    Nth[kk] = -((zpt * irt) * t1 + rpt * t2);
  }
  V2 c1D = c1[0] - c1[1], c2D = c2[0] - c2[1];
  V2 c1rD = c1[2] - c1[4], c2rD = c2[2] - c2[4];
  V2 c1zD = c1[3] - c1[5], c2zD = c2[3] - c2[5];
  const cd c3zD = c3[3] - c3[5];
  V2 Kt = ksq_mul<SIMPLE>(ap.k0sq, c2[0]) - ksq_mul<SIMPLE>(ap.k1sq, c2[1]) + iy(mr2, c1D) + iy(mr, c1rD) -
          (double(m) * m * irt2) * c2D;
  Kt.a = Kt.a + iy(mr, c3zD);
  V2 dPr = (-irt2) * c1D + irt * c1rD + c1[6] - iy(mr2, c2D) + iy(mr, c2rD);
  dPr.a = dPr.a + c3[7];
  V2 dPz = irt * c1zD + c1[7] + iy(mr, c2zD);
  dPz.a = dPz.a + c3[8];
  const V2 Kr = ksq_mul<SIMPLE>(ap.k0sq, c1[0]) - ksq_mul<SIMPLE>(ap.k1sq, c1[1]) + dPr;
  const V2 Kz = v2(ksq_mul<SIMPLE>(ap.k0sq, c3[0]) - ksq_mul<SIMPLE>(ap.k1sq, c3[1]) + dPz.a, dPz.b);
  V2 Kth = -(rpt * Kr + zpt * Kz);
  V2 EM_t = coup_mul<SIMPLE>(ap.cEM0, Nt[0]) + coup_mul<SIMPLE>(ap.cEM1, Nt[1]);
  V2 EM_th = coup_mul<SIMPLE>(ap.cEM0, Nth[0]) + coup_mul<SIMPLE>(ap.cEM1, Nth[1]);
  V2 HJ_t = coup_mul<SIMPLE>(ap.cHJ0, Nt[0]) + coup_mul<SIMPLE>(ap.cHJ1, Nt[1]);
  V2 HJ_th = coup_mul<SIMPLE>(ap.cHJ0, Nth[0]) + coup_mul<SIMPLE>(ap.cHJ1, Nth[1]);
  if (SIMPLE) {  // aEJ = 1, aHM = -1
    out[0][0] = Kt.a;   out[0][1] = Kt.b;   out[0][2] = EM_t.a;  out[0][3] = EM_t.b;
    out[1][0] = Kth.a;  out[1][1] = Kth.b;  out[1][2] = EM_th.a; out[1][3] = EM_th.b;
    out[2][0] = HJ_t.a;  out[2][1] = HJ_t.b;  out[2][2] = -Kt.a;  out[2][3] = -Kt.b;
    out[3][0] = HJ_th.a; out[3][1] = HJ_th.b; out[3][2] = -Kth.a; out[3][3] = -Kth.b;
  } else {
    out[0][0] = ap.aEJ * Kt.a;  out[0][1] = ap.aEJ * Kt.b;  out[0][2] = EM_t.a;  out[0][3] = EM_t.b;
    out[1][0] = ap.aEJ * Kth.a; out[1][1] = ap.aEJ * Kth.b; out[1][2] = EM_th.a; out[1][3] = EM_th.b;
    out[2][0] = HJ_t.a;  out[2][1] = HJ_t.b;  out[2][2] = ap.aHM * Kt.a;  out[2][3] = ap.aHM * Kt.b;
    out[3][0] = HJ_th.a; out[3][1] = HJ_th.b; out[3][2] = ap.aHM * Kth.a; out[3][3] = ap.aHM * Kth.b;
  }
}
