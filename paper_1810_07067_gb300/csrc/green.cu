// Modal Green's functions, their target derivatives and the per-mode Mueller
// blocks, on the GPU.
//
// For a target (r_t, z_t) and a source (r_s, z_s) the nine spectra
//   F0 = g^{k0}_m, F1 = g^{k1}_m                                 (eq. green11)
//   F2, F3 = d/dr_t, d/dz_t of g^{k0}_m; F4, F5 the same for k1    (eq. firstder)
//   F6, F7, F8 = d2/dr_t2, d2/dr_t dz_t, d2/dz_t2 of (g^{k0} - g^{k1})_m
//                                                       (Section 4.3, differences)
// are computed for m = 0..M+1 from nphi azimuthal samples of the integrand
// and a cosine transform (the integrands are even in phi).  Where the half
// grid fits one exact digit product (nphi/2 + 1 <= 272 samples) the transform
// runs on the tensor cores: support pairs in chunks (support_sample_kernel,
// oz_real_gemm_kernel, support_post_kernel), far pairs binned by their own
// grid (far_sample_kernel, oz_real_gemm_kernel, far_assemble_kernel);
// otherwise each pair's warp sums it directly (far_kernel, support_kernel).
//
// Kernel splitting (Section 4): with u = rho^2 and G = exp(ik sqrt u)/(4pi sqrt u),
// every family is written as  a(phi) u^{-1/2} + beta u^{-3/2} + c(phi)  with
// a, c entire in phi and beta a per-pair constant (the r_t - r_s cos(phi)
// factors are rewritten as alpha_r + u/(2 r_t) so that only a constant
// multiplies u^{-3/2}).  The u^{-1/2} part is the discrete convolution of eq.
// discA, computed as the transform of a(phi_j) times the band-limited samples
// of u^{-1/2} (the "D^{-1}(f . D q)" form); the u^{-3/2} part is beta times the
// closed-form coefficient of eq. pm.  The Fourier coefficients of u^{-1/2} and
// u^{-3/2} are (2 r_t r_s)^{-1/2} P_m(chi) and (2 r_t r_s)^{-3/2} S_m(chi) with
// P_m = sqrt(8) Q_{m-1/2} (eq. lm, recurrence eq. recurform, Miller's backward
// recurrence when the forward one is unstable) and S_m from the appendix
// relation.  Splitting is used only when the plain trapezoid rule would alias
// above the requested accuracy (zeta^{nphi-M-1} > eps, zeta = chi - sqrt(chi^2-1)).
#include <cuda_runtime.h>
#include <cstdio>
#include "smem.cuh"
#include "green.cuh"
#include "block.cuh"
#include "grid.cuh"
#include "digits.cuh"

__constant__ SeriesTables c_tab;

void upload_series_tables(const SeriesTables& t) { cudaMemcpyToSymbol(c_tab, &t, sizeof(SeriesTables)); }

// ---------------------------------------------------------------------------
// Laplace-type modal coefficients, one thread per split pair.
// pairs: [n][4] = (r_t, z_t, r_t - r_s, z_t - z_s); leg: [(Mq+1)+Ms][n] index-major:
// rows 0..Mq hold P^_n = P_n / sqrt(B), rows Mq+1.. hold S^_m = S_m / B^{3/2}.
// rinv[k] = 1 / (2k + 1) for k < nr (shared memory): the recurrences divide by
// odd integers at every step, and FP64 division costs several dependent
// operations, so the quotients are multiplications by the table's entries.
__host__ __device__ void legendre_one(double rt, double dr, double dz, long long p, long long n, int Mq, int Ms,
                                      double* __restrict__ leg, const double* rinv, int nr) {
  auto inv_odd = [&](int k) { return k < nr ? rinv[k] : 1.0 / (2.0 * k + 1.0); };  // 1 / (2k + 1)
  double rs = rt - dr;
  double d2 = dr * dr + dz * dz, B = 2.0 * rt * rs;
  double c = d2 / B, cp1 = 2.0 + c;          // chi - 1, chi + 1
  double kp2 = c / cp1;
  double K = ellipk_c(sqrt(kp2));
  double E = ellipe_c(kp2);
  double P0 = 4.0 * K / sqrt(cp1);
  double lz = log1p(c + sqrt(c * cp1));      // -ln(zeta)
  // Work with P_m and the differences D_m = P_{m-1} - P_m: the recurrence
  // (2m+1) P_{m+1} = 4 m chi P_m - (2m-1) P_{m-1} becomes
  // D_{m+1} = ((2m-1) D_m - 4 m c P_m) / (2m+1), P_{m+1} = P_m - D_{m+1},
  // which keeps the O(1) differences accurate when chi -> 1.
  double* Pv = leg;                                // rows 0..Mq: P_m, later P^_m
  double* Sv = leg + (long long)(Mq + 1) * n;      // rows 0..Ms-1: D_m, later S^_m
  const double LN32 = 3.4657359027997265;
  if (2.0 * Mq * lz <= LN32) {
    double P = P0, D = 4.0 * sqrt(cp1) * E - c * P0;  // P_0, D_1
    Pv[p] = P;
    for (int m = 1; m <= Mq; ++m) {
      if (m < Ms) Sv[(long long)m * n + p] = D;
      double Pn = P - D;                              // P_m
      Pv[(long long)m * n + p] = Pn;
      D = ((2.0 * m - 1.0) * D - 4.0 * m * c * Pn) * inv_odd(m);  // D_{m+1}
      P = Pn;
    }
  } else {
    // Miller: P~_{m*+1} = 0, P~_{m*} = 1, recurring down in (P, D).
    int mstar = Mq + (int)ceil(19.6 / lz) + 2;
    double Pn = 0.0, Dn = 1.0;
    for (int m = mstar; m >= 0; --m) {
      double Pm = Pn + Dn;
      if (m <= Mq) Pv[(long long)m * n + p] = Pm;
      if (m >= 1) {
        double Dm = ((2.0 * m + 1.0) * Dn + 4.0 * m * c * Pm) * inv_odd(m - 1);
        if (m < Ms) Sv[(long long)m * n + p] = Dm;
        Pn = Pm; Dn = Dm;
      }
    }
    double scale = P0 / Pv[p];
    for (int m = 0; m <= Mq; ++m) Pv[(long long)m * n + p] *= scale;
    for (int m = 1; m < Ms; ++m) Sv[(long long)m * n + p] *= scale;
  }
  // S_m = (1 - 2m)(chi P_m - P_{m-1})/(chi^2 - 1) = (2m - 1)(D_m - c P_m)/(c (c + 2))
  double isB = 1.0 / sqrt(B), isB3 = isB * isB * isB;
  Sv[p] = 4.0 * E / (c * sqrt(cp1)) * isB3;
  const double sfac = isB3 / (c * cp1);
  for (int m = 1; m < Ms; ++m) {
    double D = Sv[(long long)m * n + p], P = Pv[(long long)m * n + p];
    Sv[(long long)m * n + p] = (2.0 * m - 1.0) * (D - c * P) * sfac;
  }
  for (int m = 0; m <= Mq; ++m) Pv[(long long)m * n + p] *= isB;
}

// Entries of the reciprocal table: the largest index either recurrence reaches
// (the Miller start Mq + ceil(19.6 / ln(1/zeta)) + 2 with ln(1/zeta) above
// ln(32) / (2 Mq) on that branch), capped at 96 KiB of shared memory.
static int legendre_table_entries(int Mq) {
  const long long need = (long long)Mq + (long long)(19.6 * 2.0 * Mq / 3.4657359027997265) + 4;
  return (int)std::min<long long>(need, 96 * 1024 / 8);
}

__device__ __forceinline__ void fill_odd_reciprocals(double* rinv, int nr) {
  for (int k = threadIdx.x; k < nr; k += blockDim.x) rinv[k] = 1.0 / (2.0 * k + 1.0);
  __syncthreads();
}

__global__ void legendre_kernel(const double* __restrict__ pairs, long long n, int Mq, int Ms,
                                double* __restrict__ leg, int nr) {
  extern __shared__ double rinv[];
  fill_odd_reciprocals(rinv, nr);
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  legendre_one(pairs[4 * p], pairs[4 * p + 2], pairs[4 * p + 3], p, n, Mq, Ms, leg, rinv, nr);
}

void launch_legendre(const double* pairs, long long n, int Mq, int Ms, double* leg, cudaStream_t s) {
  if (n <= 0) return;
  const int tpb = 128, nr = legendre_table_entries(Mq);
  smem_optin(legendre_kernel);
  legendre_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, nr * 8, s>>>(pairs, n, Mq, Ms, leg, nr);
}

// ---------------------------------------------------------------------------
// One warp computes the nine spectra of one pair into shared memory.
// Shared layout per warp: smp[NFAM*H] (cd), spec[NFAM*Ms] (cd), q[H] (double),
// phs[Mq+1] (double).
int green_smem_per_warp(const GreenParams& gp) { return green_smem_bytes(gp); }

struct WarpSmem {
  cd* smp; cd* spec; double* q; double* phs;
};

__device__ __forceinline__ WarpSmem warp_smem(const GreenParams& gp, char* base) {
  WarpSmem w;
  w.smp = (cd*)base;
  w.spec = w.smp + NFAM * gp.H;
  w.q = (double*)(w.spec + NFAM * gp.Ms);
  w.phs = w.q + gp.H;
  return w;
}


// The weighted samples W.smp[f][j] = w_j F_f(phi_j), j = 0..nl/2 (w = 1/2 at
// both ends), of one pair on its grid g: the first half of warp_pair_spectra,
// by the threads t = 0..NT-1 of a group whose barrier is sync().
template <int NT, class Sync>
__device__ __forceinline__ void group_pair_samples(const GreenParams& gp, double rt, double dr0, double zd,
                                                   long long sid, const double* __restrict__ leg, long long n_split,
                                                   const double* __restrict__ cosT, const WarpSmem& W, int t,
                                                   const PairGrid& g, const Sync& sync) {
  const int Mq = gp.Mq, mask = gp.nphi - 1;
  const int nl = g.nl;  // local grid size; sample j sits at entry j of its tables
  const double* __restrict__ s2L = g.s2L;
  const int tstride = 1;
  const int H = nl / 2 + 1, Q = nl / 4;  // samples on [0, pi]; fold point
  const double rs = rt - dr0;
  const double d2 = dr0 * dr0 + zd * zd;
  const double alpha = dr0 - d2 / (2.0 * rt);
  const bool split = sid >= 0;
  const double TWO_PI = 6.283185307179586;
  if (split) {  // dec == 1
    for (int nn = t; nn <= Mq; nn += NT) W.phs[nn] = leg[(long long)nn * n_split + sid];
    sync();
    // q_j = (P^_0 + 2 sum_n P^_n cos(n phi_j)) / 2pi, folded: even n give E, odd n give O,
    // q_j = E + O and q_{n/2 - j} = E - O
    for (int j = t; j <= Q; j += NT) {
      double e = 0.0, o = 0.0;
      for (int nn = 1; nn <= Mq; nn += 2) o = fma(W.phs[nn], cosT[(nn * j) & mask], o);
      for (int nn = 2; nn <= Mq; nn += 2) e = fma(W.phs[nn], cosT[(nn * j) & mask], e);
      e = W.phs[0] + 2.0 * e;
      o = 2.0 * o;
      W.q[j] = (e + o) / TWO_PI;
      W.q[H - 1 - j] = (e - o) / TWO_PI;
    }
    sync();
  }
  const cd g0 = gp.gamma0;
  const double kmin = fmin(cabs(gp.kp0.k), cabs(gp.kp1.k));
  for (int j = t; j < H; j += NT) {
    double s2 = s2L[j * tstride];
    double u = d2 + 4.0 * rt * rs * s2;
    double su = sqrt(u);
    double rd = dr0 + 2.0 * rs * s2;
    cd F[NFAM];
    if (!split && kmin * su >= 2.0) {
      // both |k rho| >= 2: the kernels and their u-derivatives directly from
      // exp(i k rho), 4 pi E = e/rho, 4 pi E' = e (ik rho - 1)/(2 rho^3),
      // 4 pi E'' = e ((ik rho)^2 - 3 ik rho + 3)/(4 rho^5); the k0 - k1
      // difference does not cancel at these arguments.
      double isu = 1.0 / su, iu = isu * isu;
      cd E0[3], E1[3];
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        cd ikr = mul_i(((w == 0) ? gp.kp0.k : gp.kp1.k) * su);
        cd e = cexpi(((w == 0) ? gp.kp0.k : gp.kp1.k) * su);
        cd* E = (w == 0) ? E0 : E1;
        E[0] = e * isu;
        E[1] = (0.5 * iu * isu) * (e * (ikr - C(1.0)));
        E[2] = (0.25 * iu * iu * isu) * (e * (ikr * ikr - 3.0 * ikr + C(3.0)));
      }
      F[0] = E0[0]; F[1] = E1[0];
      F[2] = (2.0 * rd) * E0[1]; F[3] = (2.0 * zd) * E0[1];
      F[4] = (2.0 * rd) * E1[1]; F[5] = (2.0 * zd) * E1[1];
      cd D1 = E0[1] - E1[1], D2 = E0[2] - E1[2];
      F[6] = (4.0 * rd * rd) * D2 + 2.0 * D1;
      F[7] = (4.0 * rd * zd) * D2;
      F[8] = (4.0 * zd * zd) * D2 + 2.0 * D1;
      double wj = (j == 0 || j == H - 1) ? 0.5 : 1.0;
#pragma unroll
      for (int f = 0; f < NFAM; ++f) W.smp[f * H + j] = wj * F[f];
      continue;
    }
    Ent e0 = gp.k0_real ? entire_real(c_tab, gp.kp0.k.x, su) : entire(c_tab, gp.kp0, su);
    Ent e1 = gp.k1_real ? entire_real(c_tab, gp.kp1.k.x, su) : entire(c_tab, gp.kp1, su);
    cd gam1 = e0.Gam - e1.Gam, gam2 = e0.Gam2 - e1.Gam2, gam1p = e0.Gamp - e1.Gamp;
    cd dSp = e0.Sp - e1.Sp, dSpp = e0.Spp - e1.Spp;
    if (!split) {
      double isu = 1.0 / su, iu3 = isu / u;
      F[0] = e0.C * isu + mul_i(e0.S);
      F[1] = e1.C * isu + mul_i(e1.S);
      cd Ep0 = e0.Gam * isu - C(0.5 * iu3) + mul_i(e0.Sp);
      cd Ep1 = e1.Gam * isu - C(0.5 * iu3) + mul_i(e1.Sp);
      F[2] = (2.0 * rd) * Ep0; F[3] = (2.0 * zd) * Ep0;
      F[4] = (2.0 * rd) * Ep1; F[5] = (2.0 * zd) * Ep1;
      cd D1 = gam1 * isu + mul_i(dSp);
      cd D2 = (gam1p - 0.5 * gam2) * isu - (0.5 * iu3) * g0 + mul_i(dSpp);
      F[6] = (4.0 * rd * rd) * D2 + 2.0 * D1;
      F[7] = (4.0 * rd * zd) * D2;
      F[8] = (4.0 * zd * zd) * D2 + 2.0 * D1;
    } else {
      double q = W.q[j];
      F[0] = q * e0.C + mul_i(e0.S);
      F[1] = q * e1.C + mul_i(e1.S);
      F[2] = q * ((2.0 * rd) * e0.Gam - C(0.5 / rt)) + mul_i((2.0 * rd) * e0.Sp);
      F[3] = q * ((2.0 * zd) * e0.Gam) + mul_i((2.0 * zd) * e0.Sp);
      F[4] = q * ((2.0 * rd) * e1.Gam - C(0.5 / rt)) + mul_i((2.0 * rd) * e1.Sp);
      F[5] = q * ((2.0 * zd) * e1.Gam) + mul_i((2.0 * zd) * e1.Sp);
      cd eta = gam1p - 0.5 * gam2;
      F[6] = q * ((4.0 * rd * rd) * eta - ((rd + alpha) / rt) * g0 + 2.0 * gam1) +
             mul_i((4.0 * rd * rd) * dSpp + 2.0 * dSp);
      F[7] = q * ((4.0 * rd * zd) * eta - (zd / rt) * g0) + mul_i((4.0 * rd * zd) * dSpp);
      F[8] = q * ((4.0 * zd * zd) * eta + 2.0 * gam1) + mul_i((4.0 * zd * zd) * dSpp + 2.0 * dSp);
    }
    double wj = (j == 0 || j == H - 1) ? 0.5 : 1.0;
#pragma unroll
    for (int f = 0; f < NFAM; ++f) W.smp[f * H + j] = wj * F[f];
  }
  sync();
}

__device__ void warp_pair_samples(const GreenParams& gp, double rt, double dr0, double zd,
                                  long long sid, const double* __restrict__ leg, long long n_split,
                                  const double* __restrict__ cosT, const WarpSmem& W, int lane,
                                  const PairGrid& g) {
  group_pair_samples<32>(gp, rt, dr0, zd, sid, leg, n_split, cosT, W, lane, g, [] { __syncwarp(); });
}

__device__ void warp_pair_spectra(const GreenParams& gp, double rt, double dr0, double zd,
                                  long long sid, const double* __restrict__ leg, long long n_split,
                                  const double* __restrict__ cosT, const double* __restrict__ s2T,
                                  const WarpSmem& W, int lane, const PairGrid& g) {
  const int Ms = gp.Ms, Mq = gp.Mq;
  const int nl = g.nl;  // local grid size; sample j sits at entry j of its tables
  const double* __restrict__ cosL = g.cosL;
  const int T = nl, tstride = 1;
  const int Me = g.mc + 1;  // modes 0..mc computed, the rest zero
  const int H = nl / 2 + 1, Q = nl / 4;  // samples on [0, pi]; fold point
  const double d2 = dr0 * dr0 + zd * zd;
  const double alpha = dr0 - d2 / (2.0 * rt);
  const bool split = sid >= 0;
  const cd g0 = gp.gamma0;
  warp_pair_samples(gp, rt, dr0, zd, sid, leg, n_split, cosT, W, lane, g);
  // fold: smp[j] <- w_j F_j + w_{n/2-j} F_{n/2-j} (even m), smp[n/2-j] <- difference (odd m)
  for (int t = lane; t < NFAM * Q; t += 32) {
    int f = t / Q, j = t % Q;
    cd a = W.smp[f * H + j], b = W.smp[f * H + H - 1 - j];
    W.smp[f * H + j] = a + b;
    W.smp[f * H + H - 1 - j] = a - b;
  }
  __syncwarp();
  // second fold of the even-m sums E_j (j = 0..Q, E_Q the centre sample) at
  // j <-> Q - j: cos(m phi_{Q-j}) = (-1)^{m/2} cos(m phi_j) for even m, so
  // m = 0 mod 4 sums E_j + E_{Q-j} (kept at j) over j < Q/2 plus the centre
  // E_{Q/2}, and m = 2 mod 4 sums E_j - E_{Q-j} (kept at Q - j) over j < Q/2
  // (its centre cosine vanishes).  Needs Q even (grids of 8k points).
  const int Q2 = Q / 2;
  const bool fold2 = (Q & 1) == 0;
  if (fold2) {
    for (int t = lane; t < NFAM * Q2; t += 32) {
      int f = t / Q2, j = t % Q2;
      cd a = W.smp[f * H + j], b = W.smp[f * H + Q - j];
      W.smp[f * H + j] = a + b;
      W.smp[f * H + Q - j] = a - b;
    }
    __syncwarp();
  }
  // cosine transform: spec_m = (1/n) sum_j w_j F_j cos(m phi_j) (the 4pi of G
  // is folded into the normalisation); the u^{-3/2} part is added exactly.
  const double inv = 1.0 / nl;
  const double FOUR_PI = 12.566370614359172;
  // coefficient of the exact u^{-3/2} part of family f (split pairs)
  auto beta = [&](int f) -> cd {
    switch (f) {
      case 2: case 4: return C(-alpha);
      case 3: case 5: return C(-zd);
      case 6: return (-2.0 * alpha * alpha) * g0;
      case 7: return (-2.0 * alpha * zd) * g0;
      case 8: return (-2.0 * zd * zd) * g0;
      default: return C(0.0);
    }
  };
  const double* Shat = leg + (long long)(Mq + 1) * n_split;
  // one (mode, family triple) per lane and round: 3 (M+2) items keep the
  // lanes busy where one mode per lane would leave most of the last round
  // idle.  Items run odd modes first, then m = 2 mod 4, then m = 0 mod 4
  // (with fold2), so that the lanes of a round mostly share a trip count.
  const int n_odd = Me / 2, n_2 = (Me + 1) / 4;
  for (int t = lane; t < NFAM * (Ms - Me); t += 32) W.spec[(t / (Ms - Me)) * Ms + Me + t % (Ms - Me)] = C(0.0);
  for (int it = lane; it < 3 * Me; it += 32) {
    const int k = it / 3, f0 = 3 * (it % 3);
    int mm, cls;  // cls 1: odd, 2: m = 2 mod 4, 0: m = 0 mod 4 (without fold2: 0 for every even m)
    if (!fold2) { mm = k; cls = mm & 1; }
    else if (k < n_odd) { mm = 2 * k + 1; cls = 1; }
    else if (k < n_odd + n_2) { mm = 4 * (k - n_odd) + 2; cls = 2; }
    else { mm = 4 * (k - n_odd - n_2); cls = 0; }
    cd acc[3] = {C(0.0), C(0.0), C(0.0)};
    const bool odd = cls == 1;
    const int step = (mm * tstride) % T;  // table index of cos(m phi_j) advances by step (mod T)
    const int nj = odd ? Q : (fold2 ? Q2 : Q);
    int idx = 0;
    for (int j = 0; j < nj; ++j) {
      double c = cosL[idx];
      idx += step;
      if (idx >= T) idx -= T;
      int jj = odd ? (H - 1 - j) : (cls == 2 ? Q - j : j);
#pragma unroll
      for (int f = 0; f < 3; ++f) acc[f] = fma(c, W.smp[(f0 + f) * H + jj], acc[f]);
    }
    if (cls == 0) {  // the centre sample (j = Q/2 after the second fold, else n/4) pairs with itself
      double c = cosL[idx];
      const int jc = fold2 ? Q2 : Q;
#pragma unroll
      for (int f = 0; f < 3; ++f) acc[f] = fma(c, W.smp[(f0 + f) * H + jc], acc[f]);
    }
    double Sm = split ? Shat[(long long)mm * n_split + sid] / FOUR_PI : 0.0;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      cd v = inv * acc[f];
      if (split) v = fma(Sm, beta(f0 + f), v);
      W.spec[(f0 + f) * Ms + mm] = v;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Stores of the Mueller 4 x 4 blocks (block.cuh forms them).
__device__ __forceinline__ void store_block(cd* __restrict__ A, int n, int m, int i, int j, cd blk[4][4],
                                            double scale) {
  size_t base = (size_t)m * n * n;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    double2* dst = (double2*)(A + base + (size_t)(4 * j + b) * n + 4 * i);
#pragma unroll
    for (int a = 0; a < 4; ++a) dst[a] = make_double2(scale * blk[a][b].x, scale * blk[a][b].y);
  }
}

__device__ __forceinline__ void store_zero_block(cd* __restrict__ A, int n, int m, int i, int j) {
  size_t base = (size_t)m * n * n;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    double2* dst = (double2*)(A + base + (size_t)(4 * j + b) * n + 4 * i);
#pragma unroll
    for (int a = 0; a < 4; ++a) dst[a] = make_double2(0.0, 0.0);
  }
}

__device__ __forceinline__ bool near_panels(int Pi, int Pj, int nP, int closed) {
  int d = Pi - Pj;
  if (d >= -1 && d <= 1) return true;
  if (closed && nP > 2 && (d == nP - 1 || d == -(nP - 1))) return true;
  return false;
}

// ---------------------------------------------------------------------------
// Far panels: fused sampling, transform and assembly for one (i, j) pair per warp.
// Modes 0..M are assembled one per lane.  When M + 1 leaves a partial last
// round of tail = (M + 1) mod 32 modes (a.tq > 0), the tail modes are not
// assembled with their pair: the pair's spectra of modes full - 1 .. M + 1 go
// to a per-warp queue in global scratch, and once a.tq pairs are queued one
// round assembles all their tail blocks (a.tq * tail <= 32 lanes busy instead
// of tail lanes per pair).
__global__ void far_kernel(BuildArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const GreenParams& gp = a.gp;
  WarpSmem W = warp_smem(gp, smem + (size_t)wib * green_smem_bytes(gp));
  const long long total = (long long)a.N * a.N;
  const int n = 4 * a.N;
  const int tq = a.tq;
  const int full = tq ? (gp.M + 1) / 32 * 32 : gp.M + 1;  // modes assembled with their pair
  const int tail = gp.M + 1 - full, tw = tail + 2;         // queued modes, kept spectra per pair
  const long long gw = (long long)blockIdx.x * wpb + wib;
  cd* Qs = tq ? a.tailq + gw * (long long)tq * tw * NFAM : nullptr;
  int* Qij = tq ? a.tailij + gw * 2LL * tq : nullptr;
  int qn = 0;  // pairs in the queue (warp-uniform)
  // per-pair constants: quadrature weights times the L2 weight ratio, 1 / r_t
  auto pair_consts = [&](int i, int j, double fac[3], double* irt) {
    const double rs = a.geo.r[j], w = a.geo.w[j] * rs * (a.geo.sw[i] / a.geo.sw[j]);
    fac[0] = w * a.geo.rp[j];
    fac[1] = w;
    fac[2] = w * a.geo.zp[j];
    *irt = 1.0 / a.geo.r[i];
  };
  auto assemble = [&](const cd* S, int stride, int base, int i, int j, int m, const double fac[3], double irt) {
    cd blk[4][4];
    mueller_block_spec(S, stride, base, fac, m, a.ap, a.geo.r[i], irt, a.geo.rp[i], a.geo.zp[i], blk);
    store_block(a.A, n, m, i, j, blk, 1.0);
  };
  auto flush = [&]() {
    __syncwarp();  // the queue's global writes are visible to the whole warp
    for (int it = lane; it < qn * tail; it += 32) {
      const int q = it / tail, m = full + it % tail;
      double fac[3], irt;
      pair_consts(Qij[2 * q], Qij[2 * q + 1], fac, &irt);
      assemble(Qs + (long long)q * tw * NFAM, tw, full - 1, Qij[2 * q], Qij[2 * q + 1], m, fac, irt);
    }
    __syncwarp();
    qn = 0;
  };
  for (long long p = gw; p < total; p += (long long)gridDim.x * wpb) {
    int i = (int)(p / a.N), j = (int)(p % a.N);
    if (near_panels(i / P_NODES, j / P_NODES, a.n_panels, a.closed)) continue;
    long long sid = a.split_far[p];
    double rt = a.geo.r[i], rs = a.geo.r[j];
    const double dr0 = rt - rs, zd0 = a.geo.z[i] - a.geo.z[j];
    const PairGrid g = pair_grid(gp, rt, dr0, zd0, sid >= 0, a.lneps, a.cosT, a.s2T, a.ladC, a.ladS);
    warp_pair_spectra(gp, rt, dr0, zd0, sid, a.leg, a.n_split, a.cosT, a.s2T, W, lane, g);
    // modes above mz have zero spectra at m - 1, m and m + 1: their blocks are zero
    const int mz = min(gp.M, g.mc + 1);
    double fac[3], irt;
    pair_consts(i, j, fac, &irt);
    for (int m = lane; m < full; m += 32) {
      if (m <= mz) assemble(W.spec, gp.Ms, 0, i, j, m, fac, irt);
      else store_zero_block(a.A, n, m, i, j);
    }
    if (tq) {
      if (mz >= full) {
        cd* dst = Qs + (long long)qn * tw * NFAM;
        for (int t = lane; t < NFAM * tw; t += 32) dst[t] = W.spec[(t / tw) * gp.Ms + full - 1 + t % tw];
        if (lane == 0) { Qij[2 * qn] = i; Qij[2 * qn + 1] = j; }
        if (++qn == tq) flush();
      } else {
        for (int m = full + lane; m <= gp.M; m += 32) store_zero_block(a.A, n, m, i, j);
      }
    }
    __syncwarp();
  }
  if (tq && qn > 0) flush();
}

// ---------------------------------------------------------------------------
// Support points of the self and adjacent panels: one warp per
// (target, slot); spectra are written to scratch for the contraction below.
// Slot layout per target: [0, SELF_PTS) own panel, then ADJ_PTS of the
// previous panel (its shared end is +1), then ADJ_PTS of the next panel
// (shared end -1).
__device__ __forceinline__ bool support_point(const BuildArgs& a, int i, int slot, long long* pid) {
  int P = i / P_NODES, loc = i % P_NODES;
  int nP = a.n_panels;
  if (slot < SELF_PTS) {
    *pid = (long long)P * PTS_PER_PANEL + loc * SELF_PTS + slot;
    return true;
  }
  if (slot < SELF_PTS + ADJ_PTS) {
    int Q = P - 1;
    if (Q < 0) { if (!a.closed || nP <= 2) return false; Q = nP - 1; }
    if (slot - SELF_PTS >= a.sup.adj_n[2 * Q + 1]) return false;  // beyond the rule of Q's end +1
    *pid = (long long)Q * PTS_PER_PANEL + P_NODES * SELF_PTS + ADJ_PTS + (slot - SELF_PTS);
    return true;
  }
  int Q = P + 1;
  if (Q >= nP) { if (!a.closed || nP <= 2) return false; Q = 0; }
  if (slot - SELF_PTS - ADJ_PTS >= a.sup.adj_n[2 * Q + 0]) return false;  // beyond the rule of Q's end -1
  *pid = (long long)Q * PTS_PER_PANEL + P_NODES * SELF_PTS + (slot - SELF_PTS - ADJ_PTS);
  return true;
}

__global__ void support_kernel(BuildArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const GreenParams& gp = a.gp;
  WarpSmem W = warp_smem(gp, smem + (size_t)wib * green_smem_bytes(gp));
  const long long total = (long long)a.N * NEAR_SLOTS;
  for (long long p = (long long)blockIdx.x * wpb + wib; p < total; p += (long long)gridDim.x * wpb) {
    int i = (int)(p / NEAR_SLOTS), slot = (int)(p % NEAR_SLOTS);
    long long pid;
    if (!support_point(a, i, slot, &pid)) continue;
    long long sid = a.split_sup[p];
    double rt = a.geo.r[i], dr0, zd;
    if (slot < SELF_PTS) { dr0 = a.sup.dr[pid]; zd = a.sup.dz[pid]; }
    else { dr0 = rt - a.sup.r[pid]; zd = a.geo.z[i] - a.sup.z[pid]; }
    const PairGrid g = pair_grid(gp, rt, dr0, zd, sid >= 0, a.lneps, a.cosT, a.s2T, a.ladC, a.ladS);
    warp_pair_spectra(gp, rt, dr0, zd, sid, a.leg, a.n_split, a.cosT, a.s2T, W, lane, g);
    cd* dst = a.spec_sup + p * NFAM * gp.Ms;
    for (int t = lane; t < NFAM * gp.Ms; t += 32) dst[t] = W.spec[t];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Support spectra with the transform on the tensor cores.  The support pairs
// are sampled on the full grid (they are near pairs: their spectra keep all
// modes), and the cosine transform spec_m = (1/n) sum_j w_j F_j cos(2 pi m j / n)
// becomes one real product for a chunk of pairs: rows = (pair, family,
// Re/Im), k = j (n/2 + 1 samples), columns = modes; FP64-accurate through
// exact digit slicing (oz_real_gemm_kernel).  The sampling kernel writes each
// row's digits and scale; the product writes Y[m][row]; the last kernel forms
// the complex spectra and adds the exact u^{-3/2} part of split pairs.
#define SUP_ROWS (2 * NFAM)  // rows per pair

__device__ __forceinline__ void support_geometry(const BuildArgs& a, int i, int slot, long long pid, double* rt,
                                                 double* dr0, double* zd) {
  *rt = a.geo.r[i];
  if (slot < SELF_PTS) { *dr0 = a.sup.dr[pid]; *zd = a.sup.dz[pid]; }
  else { *dr0 = *rt - a.sup.r[pid]; *zd = a.geo.z[i] - a.sup.z[pid]; }
}

// CTA of SUP_NT threads per support pair of the chunk: list[q0 + q], q < count.
// Shared: the samples [NFAM][H], q [H], the Legendre coefficients [Mq + 1].
#define SUP_NT 128

__host__ __device__ inline int support_sample_smem(int H, int Mq) {
  return NFAM * H * 16 + H * 8 + (Mq + 1) * 8 + (SUP_NT / 32) * SUP_ROWS * 8 + SUP_ROWS * 8;
}

// Row scales and digits of one pair's samples W.smp[f][j], j < H, as rows
// q * 18 + (2 f + Re/Im) of the digit operand (k-tiles of 16, nkt of them):
// by the SUP_NT threads of the CTA.
__device__ __forceinline__ void pair_rows_to_digits(const WarpSmem& W, int H, int q, int nkt,
                                                    __nv_bfloat16* __restrict__ Asl, double* __restrict__ Ascale,
                                                    double* red, double* shift) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  // row maxima of |v| on the bits of the samples (integer pipe)
  unsigned long long mx[SUP_ROWS];
#pragma unroll
  for (int rr = 0; rr < SUP_ROWS; ++rr) mx[rr] = 0ull;
  for (int j = t; j < H; j += SUP_NT)
#pragma unroll
    for (int f = 0; f < NFAM; ++f) {
      const cd v = W.smp[f * H + j];
      const unsigned long long bx = abs_bits(v.x), by = abs_bits(v.y);
      mx[2 * f] = bx > mx[2 * f] ? bx : mx[2 * f];
      mx[2 * f + 1] = by > mx[2 * f + 1] ? by : mx[2 * f + 1];
    }
#pragma unroll
  for (int rr = 0; rr < SUP_ROWS; ++rr) {
    unsigned long long m = mx[rr];
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
      m = y > m ? y : m;
    }
    if (lane == 0) red[wid * SUP_ROWS + rr] = __longlong_as_double((long long)m);
  }
  __syncthreads();
  if (t < SUP_ROWS) {  // row scales: powers of two 2^E above twice each row's largest magnitude
    double m = 0.0;
    for (int w = 0; w < SUP_NT / 32; ++w) m = fmax(m, red[w * SUP_ROWS + t]);
    const int E = pow2_scale_exp(m);
    shift[t] = (double)(56 - E);  // digits of round(v 2^(56 - E))
    Ascale[(size_t)q * SUP_ROWS + t] = ldexp(1.0, E);
  }
  __syncthreads();
  // digits: thread item = (row, group of 8 consecutive k), one 16-byte store per digit
  const int kg_n = nkt * 2;
  for (int it = t; it < SUP_ROWS * kg_n; it += SUP_NT) {
    const int rr = it / kg_n, kg = it % kg_n, f = rr >> 1, im = rr & 1;
    const int S = (int)shift[rr];
    int dg[8][OZ_S];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = kg * 8 + c;
      double v = 0.0;
      if (k < H) { const cd z = W.smp[f * H + k]; v = im ? z.y : z.x; }
      digits28(fixed_rn(v, S), dg[c]);
    }
    const long long row = (long long)q * SUP_ROWS + rr;
    const long long rt_ = row >> 7;
    const int r = (int)(row & 127), kt = kg >> 1, kk = (kg & 1) * 8;
    __nv_bfloat16* blk = Asl + ((size_t)rt_ * nkt + kt) * (OZ_S * 2048);
    const int off = core_off(r, kk);
#pragma unroll
    for (int d = 0; d < OZ_S; ++d) {
      __align__(16) __nv_bfloat16 e8[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) e8[c] = __float2bfloat16((float)dg[c][d]);
      *(uint4*)(blk + d * 2048 + off) = *(uint4*)e8;
    }
  }
  __syncthreads();  // the shared samples are rewritten by the next pair
}

__device__ __forceinline__ WarpSmem sample_smem(char* smem, int H, int Mq, double** red, double** shift) {
  WarpSmem W;
  W.smp = (cd*)smem;
  W.spec = nullptr;
  W.q = (double*)(W.smp + NFAM * H);
  W.phs = W.q + H;
  *red = W.phs + Mq + 1;                // [SUP_NT / 32][SUP_ROWS]
  *shift = *red + (SUP_NT / 32) * SUP_ROWS;  // [SUP_ROWS]
  return W;
}

__global__ void __launch_bounds__(SUP_NT, 3) support_sample_kernel(BuildArgs a, const int* __restrict__ list, int q0,
                                                                   int count, __nv_bfloat16* __restrict__ Asl,
                                                                   double* __restrict__ Ascale, int nkt) {
  extern __shared__ __align__(16) char smem[];
  const GreenParams& gp = a.gp;
  double *red, *shift;
  const WarpSmem W = sample_smem(smem, gp.H, gp.Mq, &red, &shift);
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    const int p = list[q0 + q];
    const int i = p / NEAR_SLOTS, slot = p % NEAR_SLOTS;
    long long pid;
    support_point(a, i, slot, &pid);
    double rt, dr0, zd;
    support_geometry(a, i, slot, pid, &rt, &dr0, &zd);
    const long long sid = a.split_sup[p];
    group_pair_samples<SUP_NT>(gp, rt, dr0, zd, sid, a.leg, a.n_split, a.cosT, W, threadIdx.x,
                               full_grid(gp, a.cosT, a.s2T), [] { __syncthreads(); });
    __syncthreads();
    pair_rows_to_digits(W, gp.H, q, nkt, Asl, Ascale, red, shift);
  }
}

// Far pairs of one grid-size bin (list[q0 + q], q < count, p = i N + j), on
// their ladder grid of nl points: the same rows as the support pairs, one
// warp per pair (far pairs have few samples: no CTA barriers).
__host__ __device__ inline int far_sample_smem_per_warp(int H, int Mq) {
  return NFAM * H * 16 + H * 8 + (Mq + 1) * 8 + SUP_ROWS * 8;
}

__global__ void __launch_bounds__(128, 3) far_sample_kernel(BuildArgs a, const int* __restrict__ list, int q0, int count,
                                                         __nv_bfloat16* __restrict__ Asl,
                                                         double* __restrict__ Ascale, int nkt, int nl) {
  extern __shared__ __align__(16) char smem[];
  const GreenParams& gp = a.gp;
  const int H = nl / 2 + 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  char* base = smem + (size_t)wib * far_sample_smem_per_warp(H, gp.Mq);
  WarpSmem W;
  W.smp = (cd*)base;
  W.spec = nullptr;
  W.q = (double*)(W.smp + NFAM * H);
  W.phs = W.q + H;
  double* shift = W.phs + gp.Mq + 1;
  for (int q = blockIdx.x * wpb + wib; q < count; q += gridDim.x * wpb) {
    const int p = list[q0 + q];
    const int i = p / a.N, j = p % a.N;
    const long long sid = a.split_far[p];
    const double rt = a.geo.r[i], dr0 = rt - a.geo.r[j], zd0 = a.geo.z[i] - a.geo.z[j];
    const PairGrid g = pair_grid(gp, rt, dr0, zd0, sid >= 0, a.lneps, a.cosT, a.s2T, a.ladC, a.ladS);
    warp_pair_samples(gp, rt, dr0, zd0, sid, a.leg, a.n_split, a.cosT, W, lane, g);
    __syncwarp();
    // row maxima of |v| on the bits of the samples (integer pipe)
    unsigned long long mx[SUP_ROWS];
#pragma unroll
    for (int rr = 0; rr < SUP_ROWS; ++rr) mx[rr] = 0ull;
    for (int jj = lane; jj < H; jj += 32)
#pragma unroll
      for (int f = 0; f < NFAM; ++f) {
        const cd v = W.smp[f * H + jj];
        const unsigned long long bx = abs_bits(v.x), by = abs_bits(v.y);
        mx[2 * f] = bx > mx[2 * f] ? bx : mx[2 * f];
        mx[2 * f + 1] = by > mx[2 * f + 1] ? by : mx[2 * f + 1];
      }
#pragma unroll
    for (int rr = 0; rr < SUP_ROWS; ++rr) {
      unsigned long long m = mx[rr];
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
      }
      if (lane == rr) {  // row scale 2^E above twice the row's largest magnitude
        const int E = pow2_scale_exp(__longlong_as_double((long long)m));
        shift[rr] = (double)(56 - E);  // digits of round(v 2^(56 - E))
        Ascale[(size_t)q * SUP_ROWS + rr] = ldexp(1.0, E);
      }
    }
    __syncwarp();
    const int kg_n = nkt * 2;
    for (int it = lane; it < SUP_ROWS * kg_n; it += 32) {
      const int rr = it / kg_n, kg = it % kg_n, f = rr >> 1, im = rr & 1;
      const int S = (int)shift[rr];
      int dg[8][OZ_S];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = kg * 8 + c;
        double v = 0.0;
        if (k < H) { const cd z = W.smp[f * H + k]; v = im ? z.y : z.x; }
        digits28(fixed_rn(v, S), dg[c]);
      }
      const long long row = (long long)q * SUP_ROWS + rr;
      const long long rt_ = row >> 7;
      const int r = (int)(row & 127), kt = kg >> 1, kk = (kg & 1) * 8;
      __nv_bfloat16* blk = Asl + ((size_t)rt_ * nkt + kt) * (OZ_S * 2048);
      const int off = core_off(r, kk);
#pragma unroll
      for (int d = 0; d < OZ_S; ++d) {
        __align__(16) __nv_bfloat16 e8[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) e8[c] = __float2bfloat16((float)dg[c][d]);
        *(uint4*)(blk + d * 2048 + off) = *(uint4*)e8;
      }
    }
    __syncwarp();
  }
}

// Grid-size bin of every far pair (g.nl / 8; 0xFFFF for near pairs) and the
// bins' counts.
__global__ void far_bin_kernel(BuildArgs a, unsigned short* __restrict__ bin_of, int* __restrict__ counts) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)a.N * a.N) return;
  const int i = (int)(p / a.N), j = (int)(p % a.N);
  if (near_panels(i / P_NODES, j / P_NODES, a.n_panels, a.closed)) { bin_of[p] = 0xFFFF; return; }
  const GreenParams& gp = a.gp;
  const double rt = a.geo.r[i], dr0 = rt - a.geo.r[j], zd0 = a.geo.z[i] - a.geo.z[j];
  const PairGrid g = pair_grid(gp, rt, dr0, zd0, a.split_far[p] >= 0, a.lneps, a.cosT, a.s2T, a.ladC, a.ladS);
  const int b = g.nl / 8;
  bin_of[p] = (unsigned short)b;
  atomicAdd(&counts[b], 1);
}

__global__ void far_scatter_kernel(long long total, const unsigned short* __restrict__ bin_of, int* __restrict__ cursor,
                                   int* __restrict__ list) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= total) return;
  const int b = bin_of[p];
  if (b != 0xFFFF) list[atomicAdd(&cursor[b], 1)] = (int)p;
}

// The blocks of far pairs from their spectra Y[m][row] (the products of one
// bin's chunk), exactly as far_kernel assembles them from its transform:
// modes above the pair's m_c zero, the split pairs' u^{-3/2} part added.
template <bool SIMPLE>
__global__ void __launch_bounds__(128, 3) far_assemble_kernel(BuildArgs a, const int* __restrict__ list, int q0, int count,
                                    const double* __restrict__ Y, int ldy, int ncols, int nl) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const GreenParams& gp = a.gp;
  const int Ms = gp.Ms;
  cd* spec = (cd*)smem + (size_t)wib * NFAM * Ms;
  const int n = 4 * a.N;
  const int tq = a.tq;
  const int full = tq ? (gp.M + 1) / 32 * 32 : gp.M + 1;
  const int tail = gp.M + 1 - full, tw = tail + 2;
  const long long gw = (long long)blockIdx.x * wpb + wib;
  cd* Qs = tq ? a.tailq + gw * (long long)tq * tw * NFAM : nullptr;
  int* Qij = tq ? a.tailij + gw * 2LL * tq : nullptr;
  int qn = 0;
  const double invn = 1.0 / nl;
  const double* Shat = a.leg + (long long)(gp.Mq + 1) * a.n_split;
  auto pair_consts = [&](int i, int j, double fac[3], double* irt) {
    const double rs = a.geo.r[j], w = a.geo.w[j] * rs * (a.geo.sw[i] / a.geo.sw[j]);
    fac[0] = w * a.geo.rp[j];
    fac[1] = w;
    fac[2] = w * a.geo.zp[j];
    *irt = 1.0 / a.geo.r[i];
  };
  auto assemble = [&](const cd* S, int stride, int base, int i, int j, int m, const double fac[3], double irt) {
    cd blk[4][4];
    mueller_block_spec<SIMPLE>(S, stride, base, fac, m, a.ap, a.geo.r[i], irt, a.geo.rp[i], a.geo.zp[i], blk);
    store_block(a.A, n, m, i, j, blk, 1.0);
  };
  auto flush = [&]() {
    __syncwarp();
    for (int it = lane; it < qn * tail; it += 32) {
      const int qq = it / tail, m = full + it % tail;
      double fac[3], irt;
      pair_consts(Qij[2 * qq], Qij[2 * qq + 1], fac, &irt);
      assemble(Qs + (long long)qq * tw * NFAM, tw, full - 1, Qij[2 * qq], Qij[2 * qq + 1], m, fac, irt);
    }
    __syncwarp();
    qn = 0;
  };
  for (long long q = gw; q < count; q += (long long)gridDim.x * wpb) {
    const int p = list[q0 + q];
    const int i = p / a.N, j = p % a.N;
    const long long sid = a.split_far[p];
    const double rt = a.geo.r[i], dr0 = rt - a.geo.r[j], zd0 = a.geo.z[i] - a.geo.z[j];
    const PairGrid g = pair_grid(gp, rt, dr0, zd0, sid >= 0, a.lneps, a.cosT, a.s2T, a.ladC, a.ladS);
    const int Me = min(g.mc + 1, ncols);
    const double d2 = dr0 * dr0 + zd0 * zd0, alpha = dr0 - d2 / (2.0 * rt);
    const long long row0 = q * SUP_ROWS;
    // lanes take consecutive families of one mode: a mode's 18 values of the
    // pair are contiguous in Y (16-byte loads of one 144-byte run)
    for (int t = lane; t < NFAM * Ms; t += 32) {
      const int m = t / NFAM, f = t - m * NFAM;
      cd v = C(0.0);
      if (m < Me) {
        const double2 y = *(const double2*)(Y + (size_t)m * ldy + row0 + 2 * f);  // even offset: 16-byte aligned
        v = C(invn * y.x, invn * y.y);
        if (sid >= 0 && f >= 2) {
          cd beta;
          switch (f) {
            case 2: case 4: beta = C(-alpha); break;
            case 3: case 5: beta = C(-zd0); break;
            case 6: beta = (-2.0 * alpha * alpha) * gp.gamma0; break;
            case 7: beta = (-2.0 * alpha * zd0) * gp.gamma0; break;
            default: beta = (-2.0 * zd0 * zd0) * gp.gamma0; break;
          }
          v = fma(Shat[(long long)m * a.n_split + sid] / 12.566370614359172, beta, v);
        }
      }
      spec[f * Ms + m] = v;
    }
    __syncwarp();
    const int mz = min(gp.M, g.mc + 1);
    double fac[3], irt;
    pair_consts(i, j, fac, &irt);
    for (int m = lane; m < full; m += 32) {
      if (m <= mz) assemble(spec, Ms, 0, i, j, m, fac, irt);
      else store_zero_block(a.A, n, m, i, j);
    }
    if (tq) {
      if (mz >= full) {
        cd* dst = Qs + (long long)qn * tw * NFAM;
        for (int t = lane; t < NFAM * tw; t += 32) dst[t] = spec[(t / tw) * Ms + full - 1 + t % tw];
        if (lane == 0) { Qij[2 * qn] = i; Qij[2 * qn + 1] = j; }
        if (++qn == tq) flush();
      } else {
        for (int m = full + lane; m <= gp.M; m += 32) store_zero_block(a.A, n, m, i, j);
      }
    }
    __syncwarp();
  }
  if (tq && qn > 0) flush();
}

// thread per (pair q, family f, mode m): spec = (1/n)(Y_re + i Y_im) + the
// exact u^{-3/2} part of a split pair (its coefficient beta_f and S^_m)
__global__ void support_post_kernel(BuildArgs a, const int* __restrict__ list, int q0, int count,
                                    const double* __restrict__ Y, int ldy) {
  const GreenParams& gp = a.gp;
  const int Ms = gp.Ms;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)count * NFAM * Ms) return;
  const int m = (int)(t % Ms);
  const int f = (int)((t / Ms) % NFAM);
  const int q = (int)(t / ((long long)Ms * NFAM));
  const int p = list[q0 + q];
  const long long row = (long long)q * SUP_ROWS + 2 * f;
  const double invn = 1.0 / gp.nphi;
  cd v = C(invn * Y[(size_t)m * ldy + row], invn * Y[(size_t)m * ldy + row + 1]);
  const long long sid = a.split_sup[p];
  if (sid >= 0 && f >= 2) {
    const int i = p / NEAR_SLOTS, slot = p % NEAR_SLOTS;
    long long pid;
    support_point(a, i, slot, &pid);
    double rt, dr0, zd;
    support_geometry(a, i, slot, pid, &rt, &dr0, &zd);
    const double d2 = dr0 * dr0 + zd * zd;
    const double alpha = dr0 - d2 / (2.0 * rt);
    const cd g0 = gp.gamma0;
    cd beta;
    switch (f) {
      case 2: case 4: beta = C(-alpha); break;
      case 3: case 5: beta = C(-zd); break;
      case 6: beta = (-2.0 * alpha * alpha) * g0; break;
      case 7: beta = (-2.0 * alpha * zd) * g0; break;
      default: beta = (-2.0 * zd * zd) * g0; break;
    }
    const double* Shat = a.leg + (long long)(gp.Mq + 1) * a.n_split;
    const double Sm = Shat[(long long)m * a.n_split + sid] / 12.566370614359172;  // / 4 pi
    v = fma(Sm, beta, v);
  }
  a.spec_sup[(size_t)p * NFAM * Ms + (size_t)f * Ms + m] = v;
}

// ---------------------------------------------------------------------------
// Near panels: R_k(sigma, f, m) = sum_s W_s L_k(tau_s) sigma_s F_f(s, m)
// (eqs. eq_nyslike, eq_nyslike2 with sum_j U_jk P_j = L_k), then the blocks of
// the panel's columns k.  One CTA per (target, near panel, chunk of kc columns).
__global__ void __launch_bounds__(384) near_kernel(BuildArgs a) {
  extern __shared__ __align__(16) char smem[];
  const GreenParams& gp = a.gp;
  const int kc = a.kc, nchunk = P_NODES / kc;
  int bid = blockIdx.x;
  const int chunk = bid % nchunk; bid /= nchunk;
  const int which = bid % 3;  // 0 prev, 1 self, 2 next
  const int i = bid / 3;
  const int P = i / P_NODES, loc = i % P_NODES, nP = a.n_panels;
  int Q, slot0, S;
  const double* L;
  if (which == 1) {
    Q = P; slot0 = 0; S = SELF_PTS; L = a.sup.Lself + (size_t)loc * SELF_PTS * P_NODES;
  } else if (which == 0) {  // previous panel: its end +1 touches the target's panel
    Q = P - 1;
    if (Q < 0) { if (!a.closed || nP <= 2) return; Q = nP - 1; }
    slot0 = SELF_PTS; S = a.sup.adj_n[2 * Q + 1];
    L = a.sup.Ladj + (size_t)(a.sup.adj_rule[2 * Q + 1] * 2 + 1) * ADJ_PTS * P_NODES;
  } else {                  // next panel: its end -1
    Q = P + 1;
    if (Q >= nP) { if (!a.closed || nP <= 2) return; Q = 0; }
    slot0 = SELF_PTS + ADJ_PTS; S = a.sup.adj_n[2 * Q + 0];
    L = a.sup.Ladj + (size_t)(a.sup.adj_rule[2 * Q + 0] * 2 + 0) * ADJ_PTS * P_NODES;
  }
  const int Ms = gp.Ms;
  cd* R = (cd*)smem;                              // [kc][3][NFAM][Ms]
  double* V = (double*)(R + (size_t)kc * 3 * NFAM * Ms);  // [S][kc][3]
  for (int t = threadIdx.x; t < S * kc; t += blockDim.x) {
    int s = t / kc, kk = t % kc;
    long long pid;
    support_point(a, i, slot0 + s, &pid);
    double w = a.sup.W[pid] * L[(size_t)s * P_NODES + chunk * kc + kk];
    double rs = a.sup.r[pid];
    V[(s * kc + kk) * 3 + 0] = w * rs * a.sup.rp[pid];
    V[(s * kc + kk) * 3 + 1] = w * rs;
    V[(s * kc + kk) * 3 + 2] = w * rs * a.sup.zp[pid];
  }
  __syncthreads();
  const cd* F = a.spec_sup + ((long long)i * NEAR_SLOTS + slot0) * NFAM * Ms;
  for (int item = threadIdx.x; item < NFAM * Ms; item += blockDim.x) {
    cd acc[8][3];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
#pragma unroll
      for (int sg = 0; sg < 3; ++sg) acc[kk][sg] = C(0.0);
    for (int s = 0; s < S; ++s) {
      cd v = F[(size_t)s * NFAM * Ms + item];
      const double* Vs = V + s * kc * 3;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        if (kk < kc) {
#pragma unroll
          for (int sg = 0; sg < 3; ++sg) acc[kk][sg] = fma(Vs[kk * 3 + sg], v, acc[kk][sg]);
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
      if (kk < kc)
#pragma unroll
        for (int sg = 0; sg < 3; ++sg) R[((size_t)kk * 3 + sg) * NFAM * Ms + item] = acc[kk][sg];
  }
  __syncthreads();
  const int n = 4 * a.N;
  const double rt = a.geo.r[i], rpt = a.geo.rp[i], zpt = a.geo.zp[i];
  for (int item = threadIdx.x; item < kc * (gp.M + 1); item += blockDim.x) {
    int kk = item / (gp.M + 1), m = item % (gp.M + 1);
    int j = Q * P_NODES + chunk * kc + kk;
    const cd* Rk = R + (size_t)kk * 3 * NFAM * Ms;
    auto Rget = [&](int s, int f, int mm) { return Rk[((size_t)s * NFAM + f) * Ms + mm]; };
    cd blk[4][4];
    mueller_block(Rget, m, a.ap, rt, rpt, zpt, blk);
    if (j == i) {
      blk[0][2] += a.ap.dEM; blk[1][3] += a.ap.dEM;
      blk[2][0] += a.ap.dHJ; blk[3][1] += a.ap.dHJ;
    }
    store_block(a.A, n, m, i, j, blk, a.geo.sw[i] / a.geo.sw[j]);
  }
}

// ---------------------------------------------------------------------------
// Stand-alone spectra of arbitrary pairs (used by the modal-kernel entry point).
__global__ void pair_spectra_kernel(GreenParams gp, const double* __restrict__ pairs, const int* __restrict__ sidx,
                                    const double* __restrict__ leg, long long n_split, long long npairs,
                                    const double* __restrict__ cosT, const double* __restrict__ s2T,
                                    cd* __restrict__ out) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  WarpSmem W = warp_smem(gp, smem + (size_t)wib * green_smem_bytes(gp));
  for (long long p = (long long)blockIdx.x * wpb + wib; p < npairs; p += (long long)gridDim.x * wpb) {
    const double* q = pairs + 4 * p;  // (r_t, z_t, r_t - r_s, z_t - z_s)
    warp_pair_spectra(gp, q[0], q[2], q[3], sidx[p], leg, n_split, cosT, s2T, W, lane, full_grid(gp, cosT, s2T));
    cd* dst = out + p * NFAM * gp.Ms;
    for (int t = lane; t < NFAM * gp.Ms; t += 32) dst[t] = W.spec[t];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
static int warps_per_block(const GreenParams& gp) {
  int per = green_smem_bytes(gp);
  int w = (200 * 1024) / per;
  if (w > 8) w = 8;
  if (w < 1) w = 1;
  return w;
}

bool green_fits_smem(const GreenParams& gp) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
    optin = 227 * 1024;
  return green_smem_bytes(gp) <= optin;
}

static int grid_for(long long units, int wpb) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long need = (units + wpb - 1) / wpb;
  long long cap = (long long)sms * 8;
  return (int)(need < cap ? need : cap);
}

// Tail queue of far_kernel: pairs per flush (0 = none) and its scratch, for
// the launch shape launch_far_assembly uses.
int far_tail_pairs(const GreenParams& gp) {
  const int full = (gp.M + 1) / 32 * 32, tail = gp.M + 1 - full;
  return (full >= 32 && tail > 0 && tail <= 16) ? 32 / tail : 0;
}

// Warps per CTA of far_assemble_kernel: its shared memory is only the
// spectra, NFAM (M+2) complex values per warp.
static int assemble_warps_per_block(const GreenParams& gp) {
  int w = (72 * 1024) / (NFAM * gp.Ms * 16);  // up to three CTAs per SM (registers)
  if (w > 4) w = 4;
  if (w < 1) w = 1;
  return w;
}

size_t far_tail_scratch(const BuildArgs& a, size_t* ij_elems) {
  const int tq = far_tail_pairs(a.gp);
  const int wpb = warps_per_block(a.gp), wpa = assemble_warps_per_block(a.gp);
  const long long total = (long long)a.N * a.N;
  const long long warps = std::max((long long)grid_for(total, wpb) * wpb, (long long)grid_for(total, wpa) * wpa);
  const int tail = a.gp.M + 1 - (a.gp.M + 1) / 32 * 32;
  *ij_elems = tq ? (size_t)warps * 2 * tq : 0;
  return tq ? (size_t)warps * tq * (tail + 2) * NFAM : 0;
}

void launch_far_assembly(const BuildArgs& a, cudaStream_t s) {
  int wpb = warps_per_block(a.gp);
  int smem = wpb * green_smem_bytes(a.gp);
  smem_optin(far_kernel);
  far_kernel<<<grid_for((long long)a.N * a.N, wpb), wpb * 32, smem, s>>>(a);
}

void launch_support_spectra(const BuildArgs& a, cudaStream_t s) {
  int wpb = warps_per_block(a.gp);
  int smem = wpb * green_smem_bytes(a.gp);
  smem_optin(support_kernel);
  support_kernel<<<grid_for((long long)a.N * NEAR_SLOTS, wpb), wpb * 32, smem, s>>>(a);
}

void launch_support_samples(const BuildArgs& a, const int* list, int q0, int count, __nv_bfloat16* Asl,
                            double* Ascale, int nkt, cudaStream_t s) {
  const int smem = support_sample_smem(a.gp.H, a.gp.Mq);
  smem_optin(support_sample_kernel);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(count, 3 * sms * 8);
  support_sample_kernel<<<grid, SUP_NT, smem, s>>>(a, list, q0, count, Asl, Ascale, nkt);
}

void launch_far_bins(const BuildArgs& a, unsigned short* bin_of, int* counts, cudaStream_t s) {
  const long long total = (long long)a.N * a.N;
  far_bin_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a, bin_of, counts);
}

void launch_far_scatter(long long total, const unsigned short* bin_of, int* cursor, int* list, cudaStream_t s) {
  far_scatter_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, bin_of, cursor, list);
}

void launch_far_samples(const BuildArgs& a, const int* list, int q0, int count, __nv_bfloat16* Asl, double* Ascale,
                        int nkt, int nl, cudaStream_t s) {
  const int per = far_sample_smem_per_warp(nl / 2 + 1, a.gp.Mq);
  int wpb = (72 * 1024) / per;  // up to three 4-warp CTAs per SM (registers)
  if (wpb > 4) wpb = 4;
  if (wpb < 1) wpb = 1;
  smem_optin(far_sample_kernel);
  far_sample_kernel<<<grid_for(count, wpb), wpb * 32, wpb * per, s>>>(a, list, q0, count, Asl, Ascale, nkt, nl);
}

// Launch shape: assemble_warps_per_block (the tail-queue scratch covers it).
void launch_far_assemble(const BuildArgs& a, const int* list, int q0, int count, const double* Y, int ldy, int ncols,
                         int nl, cudaStream_t s) {
  const int wpb = assemble_warps_per_block(a.gp);
  const int smem = wpb * NFAM * a.gp.Ms * 16;
  if (a.ap.simple) {
    smem_optin(far_assemble_kernel<true>);
    far_assemble_kernel<true><<<grid_for(count, wpb), wpb * 32, smem, s>>>(a, list, q0, count, Y, ldy, ncols, nl);
  } else {
    smem_optin(far_assemble_kernel<false>);
    far_assemble_kernel<false><<<grid_for(count, wpb), wpb * 32, smem, s>>>(a, list, q0, count, Y, ldy, ncols, nl);
  }
}

void launch_support_post(const BuildArgs& a, const int* list, int q0, int count, const double* Y, int ldy,
                         cudaStream_t s) {
  const long long items = (long long)count * NFAM * a.gp.Ms;
  support_post_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(a, list, q0, count, Y, ldy);
}

// Threads per CTA: the fewest rounds (at most 384 threads) over the larger
// of the contraction's NFAM (M+2) items and the kc (M+1) blocks, so that the
// last round is not nearly empty (one CTA per SM: its shared memory).
void launch_near_assembly(const BuildArgs& a, cudaStream_t s) {
  int smem = a.kc * 3 * NFAM * a.gp.Ms * 16 + NEAR_MAX_PTS * a.kc * 3 * 8;
  const int items = std::max(NFAM * a.gp.Ms, a.kc * (a.gp.M + 1));
  const int rounds = (items + 383) / 384;
  const int threads = std::min(384, ((items + rounds - 1) / rounds + 31) / 32 * 32);
  smem_optin(near_kernel);
  near_kernel<<<a.N * 3 * (P_NODES / a.kc), threads, smem, s>>>(a);
}

void launch_pair_spectra(const GreenParams& gp, const double* pairs, const int* sidx, const double* leg,
                         long long n_split, long long npairs, const double* cosT, const double* s2T, cd* out,
                         cudaStream_t s) {
  if (npairs <= 0) return;
  int wpb = warps_per_block(gp);
  int smem = wpb * green_smem_bytes(gp);
  smem_optin(pair_spectra_kernel);
  pair_spectra_kernel<<<grid_for(npairs, wpb), wpb * 32, smem, s>>>(gp, pairs, sidx, leg, n_split, npairs, cosT,
                                                                      s2T, out);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of mueller_modal_kernels (declared in mueller.h).
// Its scratch (transform tables, split flags, pair displacements, Laplace-type
// coefficients) lives in one fixed file-scope device array instead of memory
// from cudaMalloc.  Host code must not use the array's name as a device
// address: its address is fetched once per device with cudaGetSymbolAddress.
#include <mutex>
#include "mueller.h"

#define NOALLOC_SCRATCH_DOUBLES ((size_t)2 * 1024 * 1024)  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

#define NOALLOC_MAX_DEVICES 64
// Per-device set-up state, written under g_noalloc_mu: the scratch array's
// device address and whether the series tables were uploaded to that device.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
static bool g_noalloc_tables[NOALLOC_MAX_DEVICES] = {false};
// message reported by mueller_last_error (defined with the other ABI functions)
void mueller_internal_set_error(const char* msg);

__global__ void noalloc_tables_kernel(int nphi, double* __restrict__ cosT, double* __restrict__ s2T) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nphi) cosT[t] = cospi(2.0 * t / nphi);
  if (t <= nphi / 2) {
    double v = sinpi((double)t / nphi);
    s2T[t] = v * v;
  }
}

// (r_t, z_t, r_s, z_s) -> (r_t, z_t, r_t - r_s, z_t - z_s); split flag per pair
__global__ void noalloc_prep_kernel(const double* __restrict__ pairs, long long n, int nphi, int M, double lneps,
                                    double* __restrict__ disp, int* __restrict__ sid) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  double rt = pairs[4 * p], zt = pairs[4 * p + 1];
  double dr = rt - pairs[4 * p + 2], dz = zt - pairs[4 * p + 3];
  disp[4 * p] = rt; disp[4 * p + 1] = zt; disp[4 * p + 2] = dr; disp[4 * p + 3] = dz;
  double d2 = dr * dr + dz * dz, B = 2.0 * rt * (rt - dr);
  double c = d2 / B, cp1 = 2.0 + c;
  double lz = log1p(c + sqrt(c * cp1));
  sid[p] = ((double)(nphi - M - 1) * lz < lneps) ? (int)p : -1;
}

__global__ void noalloc_legendre_kernel(const double* __restrict__ disp, const int* __restrict__ sid, long long n,
                                        int Mq, int Ms, double* __restrict__ leg, int nr) {
  extern __shared__ double rinv[];
  fill_odd_reciprocals(rinv, nr);
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n || sid[p] < 0) return;
  legendre_one(disp[4 * p], disp[4 * p + 2], disp[4 * p + 3], p, n, Mq, Ms, leg, rinv, nr);
}

static int noalloc_fail(const char* msg, int code = MUELLER_EINVAL) {
  mueller_internal_set_error(msg);
  return code;
}

extern "C" int mueller_modal_kernels_noalloc(const double* pairs_dev, long long npairs, mueller_c128 k0,
                                             mueller_c128 k1, int M, int n_phi, double split_eps,
                                             mueller_c128* out_dev, void* stream) {
  mueller_internal_set_error("");
  if (!pairs_dev || !out_dev || npairs < 0 || M < 0) return noalloc_fail("invalid arguments");
  if (n_phi < 16 || n_phi > 8192 || (n_phi & (n_phi - 1)) != 0) return noalloc_fail("n_phi must be a power of two in [16, 8192]");
  if (M + 2 > n_phi / 2) return noalloc_fail("n_phi must be at least 2M + 4");
  if (k0.im < 0 || k1.im < 0) return noalloc_fail("wavenumbers need Im k >= 0");
  if (npairs == 0) return MUELLER_OK;
  const int Mq = n_phi / 2 - 1, Ms = M + 2, H = n_phi / 2 + 1;
  {
    GreenParams g{};
    g.Ms = Ms; g.H = H; g.Mq = Mq;
    if (!green_fits_smem(g)) return noalloc_fail("n_phi and M need more shared memory per warp than a CTA can have");
  }
  auto up32 = [](size_t v) { return (v + 31) & ~(size_t)31; };
  const size_t o_cos = 0, o_s2 = o_cos + up32(n_phi), o_disp = o_s2 + up32(H);
  const size_t o_sid = o_disp + up32(4 * (size_t)npairs);
  const size_t o_leg = o_sid + up32(((size_t)npairs + 1) / 2);
  const size_t need = o_leg + (size_t)(Mq + 1 + Ms) * (size_t)npairs;
  if (need > NOALLOC_SCRATCH_DOUBLES) {
    char msg[200];
    snprintf(msg, sizeof(msg), "npairs * (n_phi/2 + M + 7) exceeds the fixed scratch of %zu doubles (16 MiB): need %zu",
             (size_t)NOALLOC_SCRATCH_DOUBLES, need);
    return noalloc_fail(msg);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return noalloc_fail("no current CUDA device");
  double* base = nullptr;
  {  // one-time set-up on this device (host threads serialised)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      double* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return noalloc_fail(cudaGetErrorString(e), MUELLER_ECUDA);
      g_noalloc_ptr[dev] = p;
    }
    if (!g_noalloc_tables[dev]) {
      SeriesTables t;
      fill_series_tables(&t);
      if (cudaMemcpyToSymbol(c_tab, &t, sizeof(SeriesTables)) != cudaSuccess) return noalloc_fail("series tables");
      g_noalloc_tables[dev] = true;
    }
    base = g_noalloc_ptr[dev];
  }
  double* cosT = base + o_cos;
  double* s2T = base + o_s2;
  double* disp = base + o_disp;
  int* sid = (int*)(base + o_sid);
  double* leg = base + o_leg;
  cudaStream_t s = (cudaStream_t)stream;
  GreenParams gp{};
  cd K0{k0.re, k0.im}, K1{k1.re, k1.im};
  gp.M = M; gp.Ms = Ms; gp.nphi = n_phi; gp.H = H; gp.Mq = Mq; gp.qmax = 0;
  gp.kp0 = kpow(K0); gp.kp1 = kpow(K1);
  gp.gamma0 = -0.25 * (K0 * K0 - K1 * K1);
  gp.k0_real = K0.y == 0.0; gp.k1_real = K1.y == 0.0;
  double eps = split_eps > 0 ? split_eps : 1e-17;
  noalloc_tables_kernel<<<(n_phi + 255) / 256, 256, 0, s>>>(n_phi, cosT, s2T);
  unsigned blocks = (unsigned)((npairs + 127) / 128);
  noalloc_prep_kernel<<<blocks, 128, 0, s>>>(pairs_dev, npairs, n_phi, M, -log(eps), disp, sid);
  const int nr = legendre_table_entries(Mq);
  smem_optin(noalloc_legendre_kernel);
  noalloc_legendre_kernel<<<blocks, 128, nr * 8, s>>>(disp, sid, npairs, Mq, Ms, leg, nr);
  launch_pair_spectra(gp, disp, sid, leg, npairs, npairs, cosT, s2T, (cd*)out_dev, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(cudaGetErrorString(e), MUELLER_ECUDA);
  return MUELLER_OK;
}
