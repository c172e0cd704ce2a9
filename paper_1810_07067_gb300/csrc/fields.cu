// Incident data and far fields (Section 6).
#include "smem.cuh"
#include "fields.cuh"

// One CTA per (node, wave): samples of the tangential traces on the node's
// ring at n_theta azimuths, then their Fourier coefficients for m = -M..M.
// Fourier coefficients (1/n_theta) sum_t s_t e^{-i m theta_t} of the four ring
// traces smp[n_theta][4] (twiddles tw[t] = e^{-2 pi i t/n_theta}), scaled by
// sE (rows 0, 1) and sH (rows 2, 3).  With n_theta = 2^L q (L <= 4), L
// decimation-in-frequency stages first split each row into 2^L sub-sequences
// of q samples (block bitrev(m mod 2^L) holds the terms of the modes of that
// residue, twiddled), so each mode is a q-term sum instead of n_theta terms;
// then one (mode, row) per thread.  Called by every thread of the CTA;
// smp is overwritten.
__device__ void modal_dft(cd* smp, const cd* tw, int n_theta, int M, int nrhs, int w, int i, int n, cd sE,
                          cd sH, cd* __restrict__ rhs) {
  int L = 0;
  while (L < 4 && ((n_theta >> L) & 1) == 0) ++L;
  for (int st = 0, len = n_theta; st < L; ++st, len >>= 1) {
    const int half = len >> 1, tstep = n_theta / len;
    for (int item = threadIdx.x; item < 4 * (n_theta >> 1); item += blockDim.x) {
      const int a = item & 3, bt = item >> 2;             // row, butterfly
      const int blk = bt / half, t = bt % half;
      const int i0 = blk * len + t, i1 = i0 + half;
      const cd u = smp[4 * i0 + a], v = smp[4 * i1 + a];
      smp[4 * i0 + a] = u + v;
      smp[4 * i1 + a] = (u - v) * tw[t * tstep];
    }
    __syncthreads();
  }
  const int q = n_theta >> L, mask = (1 << L) - 1;
  const double inv = 1.0 / n_theta;
  for (int item = threadIdx.x; item < 4 * (2 * M + 1); item += blockDim.x) {
    const int mq = item >> 2, a = item & 3;
    const int m = mq - M;
    const int mm = ((m % n_theta) + n_theta) % n_theta;
    const int r = mm & mask;
    int blk = 0;
    for (int bit = 0; bit < L; ++bit) blk |= ((r >> bit) & 1) << (L - 1 - bit);
    const int step = (mm >> L) << L;  // twiddle index advance: (mm >> L) 2^L (mod n_theta)
    const cd* x = smp + 4 * blk * q;
    cd acc = C(0.0);
    int idx = 0;
    for (int t = 0; t < q; ++t) {
      acc = fma(x[4 * t + a], tw[idx], acc);
      idx += step;
      if (idx >= n_theta) idx -= n_theta;
    }
    rhs[((size_t)mq * nrhs + w) * n + 4 * i + a] = (a < 2 ? sE : sH) * (inv * acc);
  }
}

// n x v = v_theta t - v_t e_theta at one ring point: (v_theta, -v_t)
__device__ __forceinline__ void traces(const cd v[3], double ct, double st, double rp, double zp, cd* out2) {
  cd vr = ct * v[0] + st * v[1], vth = ct * v[1] - st * v[0];
  out2[0] = vth;
  out2[1] = -(rp * vr + zp * v[2]);
}

__global__ void rhs_kernel(FieldGeom g, int M, cd k0, double omega, cd mu0, cd sE, cd sH,
                           const double* __restrict__ dirs, const double* __restrict__ pols, int nrhs, int n_theta,
                           cd* __restrict__ rhs) {
  extern __shared__ __align__(16) char smem[];
  cd* smp = (cd*)smem;         // [n_theta][4]
  cd* tw = smp + 4 * n_theta;  // [n_theta]: e^{-2 pi i t / n_theta}
  const int i = blockIdx.x, w = blockIdx.y;
  const double* d = dirs + 3 * w;
  const double* e = pols + 3 * w;
  // H polarisation (k0/(omega mu0)) d x e
  cd hf = k0 / (omega * mu0);
  double hx = d[1] * e[2] - d[2] * e[1], hy = d[2] * e[0] - d[0] * e[2], hz = d[0] * e[1] - d[1] * e[0];
  const double r = g.r[i], z = g.z[i], rp = g.rp[i], zp = g.zp[i];
  for (int t = threadIdx.x; t < n_theta; t += blockDim.x) {
    double ct, st;
    sincospi(2.0 * t / n_theta, &st, &ct);
    tw[t] = C(ct, -st);
    double phase = r * (d[0] * ct + d[1] * st) + z * d[2];
    cd ph = cexpi(k0 * phase);
    cd hph = hf * ph;
    const cd E[3] = {e[0] * ph, e[1] * ph, e[2] * ph};
    const cd H[3] = {hx * hph, hy * hph, hz * hph};
    traces(E, ct, st, rp, zp, smp + 4 * t);
    traces(H, ct, st, rp, zp, smp + 4 * t + 2);
  }
  __syncthreads();
  modal_dft(smp, tw, n_theta, M, nrhs, w, i, 4 * g.N, sE, sH, rhs);
}

// Sampled incident fields EH[w][i][t][6] (E then H, Cartesian) at the ring
// points of node i -> modal data, as rhs_kernel.
__global__ void rhs_samples_kernel(FieldGeom g, int M, cd sE, cd sH, const cd* __restrict__ EH, int nrhs,
                                   int n_theta, cd* __restrict__ rhs) {
  extern __shared__ __align__(16) char smem[];
  cd* smp = (cd*)smem;
  cd* tw = smp + 4 * n_theta;
  const int i = blockIdx.x, w = blockIdx.y;
  const double rp = g.rp[i], zp = g.zp[i];
  const cd* src = EH + ((size_t)w * g.N + i) * n_theta * 6;
  for (int t = threadIdx.x; t < n_theta; t += blockDim.x) {
    double ct, st;
    sincospi(2.0 * t / n_theta, &st, &ct);
    tw[t] = C(ct, -st);
    traces(src + 6 * t, ct, st, rp, zp, smp + 4 * t);
    traces(src + 6 * t + 3, ct, st, rp, zp, smp + 4 * t + 2);
  }
  __syncthreads();
  modal_dft(smp, tw, n_theta, M, nrhs, w, i, 4 * g.N, sE, sH, rhs);
}

void launch_rhs_samples(const FieldGeom& g, int M, cd sE, cd sH, const cd* EH, int nrhs, int n_theta, cd* rhs,
                        cudaStream_t s) {
  int smem = n_theta * 5 * (int)sizeof(cd);
  smem_optin(rhs_samples_kernel);
  rhs_samples_kernel<<<dim3(g.N, nrhs), 256, smem, s>>>(g, M, sE, sH, EH, nrhs, n_theta, rhs);
}

void launch_rhs_planewave(const FieldGeom& g, int M, cd k0, double omega, cd mu0, cd sE, cd sH,
                          const double* dirs_dev, const double* pols_dev, int nrhs, int n_theta, cd* rhs,
                          cudaStream_t s) {
  int smem = n_theta * 5 * (int)sizeof(cd);
  smem_optin(rhs_kernel);
  rhs_kernel<<<dim3(g.N, nrhs), 256, smem, s>>>(g, M, k0, omega, mu0, sE, sH, dirs_dev, pols_dev, nrhs, n_theta,
                                                 rhs);
}

// Currents on the node rings: cur[w][i][t][a] = sum_m x[m][w][4i+a] e^{i m theta_t}.
__global__ void ring_kernel(int N, int M, const cd* __restrict__ x, int nrhs, int n_theta, cd* __restrict__ cur) {
  const int i = blockIdx.x, w = blockIdx.y;
  const int n = 4 * N;
  for (int t = threadIdx.x; t < n_theta; t += blockDim.x) {
    cd acc[4] = {C(0.0), C(0.0), C(0.0), C(0.0)};
    for (int mq = 0; mq < 2 * M + 1; ++mq) {
      int m = mq - M;
      int mm = ((m % n_theta) + n_theta) % n_theta;
      int idx = (int)(((long long)mm * t) % n_theta);
      double s, c;
      sincospi(2.0 * idx / n_theta, &s, &c);
      cd ex = C(c, s);
      const cd* xv = x + ((size_t)mq * nrhs + w) * n + 4 * i;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fma(xv[a], ex, acc[a]);
    }
    cd* dst = cur + (((size_t)w * N + i) * n_theta + t) * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a) dst[a] = acc[a];
  }
}

// One CTA per (rhs, direction): Jh, Mh by the ring quadrature, then E_oo.
__global__ void farfield_kernel(FieldGeom g, cd k0, double omega, cd eps0, const cd* __restrict__ cur, int nrhs,
                                const double* __restrict__ dirs, int ndir, int n_theta, cd* __restrict__ E) {
  const int dix = blockIdx.x, w = blockIdx.y;
  const double xh0 = dirs[3 * dix], xh1 = dirs[3 * dix + 1], xh2 = dirs[3 * dix + 2];
  cd J[3] = {C(0.0), C(0.0), C(0.0)}, Mv[3] = {C(0.0), C(0.0), C(0.0)};
  const long long total = (long long)g.N * n_theta;
  const double TWO_PI = 6.283185307179586;
  for (long long it = threadIdx.x; it < total; it += blockDim.x) {
    int i = (int)(it / n_theta), t = (int)(it % n_theta);
    double s, c;
    sincospi(2.0 * t / n_theta, &s, &c);
    double r = g.r[i], z = g.z[i];
    double proj = xh0 * r * c + xh1 * r * s + xh2 * z;
    double da = g.w[i] * r * (TWO_PI / n_theta);
    cd ph = da * cexpi(-(k0 * proj));
    const cd* cv = cur + (((size_t)w * g.N + i) * n_theta + t) * 4;
    // t = r' e_r + z' e_z ; e_theta = (-s, c, 0)
    double tx = g.rp[i] * c, ty = g.rp[i] * s, tz = g.zp[i];
    cd j1 = ph * cv[0], j2 = ph * cv[1], m1 = ph * cv[2], m2 = ph * cv[3];
    J[0] += tx * j1 - s * j2; J[1] += ty * j1 + c * j2; J[2] += tz * j1;
    Mv[0] += tx * m1 - s * m2; Mv[1] += ty * m1 + c * m2; Mv[2] += tz * m1;
  }
  __shared__ cd red[6][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  cd vals[6] = {J[0], J[1], J[2], Mv[0], Mv[1], Mv[2]};
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      vals[a].x += __shfl_xor_sync(0xffffffffu, vals[a].x, o);
      vals[a].y += __shfl_xor_sync(0xffffffffu, vals[a].y, o);
    }
    if (lane == 0) red[a][wid] = vals[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cd tot[6];
    for (int a = 0; a < 6; ++a) {
      tot[a] = C(0.0);
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot[a] += red[a][q];
    }
    cd xJ = xh0 * tot[0] + xh1 * tot[1] + xh2 * tot[2];
    cd pre = -(k0 * k0) / (C(0.0, omega) * eps0);
    double xh[3] = {xh0, xh1, xh2};
    cd cr[3];
    cr[0] = xh1 * tot[5] - xh2 * tot[4];
    cr[1] = xh2 * tot[3] - xh0 * tot[5];
    cr[2] = xh0 * tot[4] - xh1 * tot[3];
    cd ik = mul_i(k0);
    double inv4pi = 1.0 / (4.0 * 3.141592653589793);
    cd* dst = E + ((size_t)w * ndir + dix) * 3;
    for (int a = 0; a < 3; ++a) dst[a] = inv4pi * (pre * (tot[a] - xh[a] * xJ) + ik * cr[a]);
  }
}

void launch_far_field(const FieldGeom& g, int M, cd k0, double omega, cd eps0, const cd* x, int nrhs,
                      const double* dirs_dev, int ndir, int n_theta, cd* cur, cd* E, cudaStream_t s) {
  ring_kernel<<<dim3(g.N, nrhs), 128, 0, s>>>(g.N, M, x, nrhs, n_theta, cur);
  farfield_kernel<<<dim3(ndir, nrhs), 256, 0, s>>>(g, k0, omega, eps0, cur, nrhs, dirs_dev, ndir, n_theta, E);
}

// ---------------------------------------------------------------------------
// Fields at points off the surface: E = cJ curl curl S J + cM curl S M,
// H = dM curl curl S M + dJ curl S J (eqs. exteriorfield, interiorfield,
// interior_dual with the region's constants), with
//   curl S V      = sum G (ik - 1/R) Rh x V da,
//   curl curl S V = sum G [(k^2 + ik/R - 1/R^2) V + (-k^2 - 3ik/R + 3/R^2)(Rh.V) Rh] da
// over the node rings (ds-weights x trapezoid in theta).  One CTA per
// (point, right-hand side); ring currents cur[w][i][t][4] from ring_kernel.
__global__ void __launch_bounds__(256) nearfield_kernel(FieldGeom g, int n_theta, const cd* __restrict__ cur,
                                                        const double* __restrict__ X, int nt, int nrhs, cd k,
                                                        cd cJ, cd cM, cd dM, cd dJ, cd* __restrict__ out) {
  const int p = blockIdx.x, w = blockIdx.y;
  const double x0 = X[3 * p], x1 = X[3 * p + 1], x2 = X[3 * p + 2];
  cd acc[12];  // curl curl S J, curl S M, curl curl S M, curl S J (3 components each)
#pragma unroll
  for (int a = 0; a < 12; ++a) acc[a] = C(0.0);
  const cd ik = mul_i(k), k2 = k * k;
  const double FOUR_PI = 12.566370614359172, TWO_PI = 6.283185307179586;
  const long long total = (long long)g.N * n_theta;
  for (long long it = threadIdx.x; it < total; it += blockDim.x) {
    const int i = (int)(it / n_theta), t = (int)(it % n_theta);
    double s, c;
    sincospi(2.0 * t / n_theta, &s, &c);
    const double r = g.r[i], z = g.z[i];
    const double tx = g.rp[i] * c, ty = g.rp[i] * s, tz = g.zp[i];  // unit tangent; e_theta = (-s, c, 0)
    const cd* cv = cur + (((size_t)w * g.N + i) * n_theta + t) * 4;
    const cd J[3] = {tx * cv[0] - s * cv[1], ty * cv[0] + c * cv[1], tz * cv[0]};
    const cd Mv[3] = {tx * cv[2] - s * cv[3], ty * cv[2] + c * cv[3], tz * cv[2]};
    const double R0 = x0 - r * c, R1 = x1 - r * s, R2 = x2 - z;
    const double R = sqrt(R0 * R0 + R1 * R1 + R2 * R2), iR = 1.0 / R;
    const double h0 = R0 * iR, h1 = R1 * iR, h2 = R2 * iR;
    const double da = g.w[i] * r * (TWO_PI / n_theta);
    const cd G = (da * iR / FOUR_PI) * cexpi(k * R);
    const cd c1 = G * (ik - C(iR));
    const cd aa = G * (k2 + iR * ik - C(iR * iR));
    const cd bb = G * (C(3.0 * iR * iR) - k2 - (3.0 * iR) * ik);
    const cd pJ = h0 * J[0] + h1 * J[1] + h2 * J[2];
    const cd pM = h0 * Mv[0] + h1 * Mv[1] + h2 * Mv[2];
    const double hv[3] = {h0, h1, h2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      acc[d] += aa * J[d] + (bb * pJ) * hv[d];
      acc[6 + d] += aa * Mv[d] + (bb * pM) * hv[d];
    }
    acc[3] += c1 * (h1 * Mv[2] - h2 * Mv[1]);
    acc[4] += c1 * (h2 * Mv[0] - h0 * Mv[2]);
    acc[5] += c1 * (h0 * Mv[1] - h1 * Mv[0]);
    acc[9] += c1 * (h1 * J[2] - h2 * J[1]);
    acc[10] += c1 * (h2 * J[0] - h0 * J[2]);
    acc[11] += c1 * (h0 * J[1] - h1 * J[0]);
  }
  __shared__ cd red[12][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      acc[a].x += __shfl_xor_sync(0xffffffffu, acc[a].x, o);
      acc[a].y += __shfl_xor_sync(0xffffffffu, acc[a].y, o);
    }
    if (lane == 0) red[a][wid] = acc[a];
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    cd tot = C(0.0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[threadIdx.x][q];
    red[threadIdx.x][0] = tot;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int d = threadIdx.x % 3;
    cd v = (threadIdx.x < 3) ? cJ * red[d][0] + cM * red[3 + d][0] : dM * red[6 + d][0] + dJ * red[9 + d][0];
    out[((size_t)w * nt + p) * 6 + threadIdx.x] = v;
  }
}

void launch_near_field(const FieldGeom& g, int M, const cd* x, int nrhs, const double* X_dev, int nt, int n_theta,
                       cd k, cd cJ, cd cM, cd dM, cd dJ, cd* cur, cd* out, cudaStream_t s) {
  ring_kernel<<<dim3(g.N, nrhs), 128, 0, s>>>(g.N, M, x, nrhs, n_theta, cur);
  nearfield_kernel<<<dim3(nt, nrhs), 256, 0, s>>>(g, n_theta, cur, X_dev, nt, nrhs, k, cJ, cM, dM, dJ, out);
}

// ---------------------------------------------------------------------------
// Far field on a (polar x azimuth) grid, mode by mode.  For x_hat at polar
// angle theta and azimuth phi, substituting theta' = phi + alpha on each ring
// turns eq. farfieldform into E(theta, phi) = R_z(phi) sum_m e^{i m phi} F_m(theta),
// with F_m the far-field vector of mode m in the frame (e_rho, e_phi, e_z) of
// azimuth phi, where x_hat = (sin theta, 0, cos theta).  The ring integrals
// need c_m = (1/n) sum_t e^{-i a cos alpha_t} e^{i m alpha_t}, a = k0 r sin theta
// (same trapezoid rule in alpha as mueller_far_field):
//   (1/2pi) int e^{-i a cos} e^{i m alpha} {1, cos, sin} = {c_m, (c_{m+1}+c_{m-1})/2, (c_{m+1}-c_{m-1})/(2i)}.

// coef[p][j][m + M + 1], |m| <= M + 1: one CTA per (polar angle, node)
__global__ void ffgrid_coef_kernel(FieldGeom g, int M, cd k0, int n_polar, int n_alpha, cd* __restrict__ coef) {
  extern __shared__ __align__(16) char smem[];
  cd* f = (cd*)smem;           // [n_alpha]
  cd* tw = f + n_alpha;        // [n_alpha] e^{+2 pi i t / n_alpha}
  const int p = blockIdx.x, j = blockIdx.y;
  double sth, cth;
  sincospi((p + 0.5) / n_polar, &sth, &cth);
  const cd a = (g.r[j] * sth) * k0;
  for (int t = threadIdx.x; t < n_alpha; t += blockDim.x) {
    double s, c;
    sincospi(2.0 * t / n_alpha, &s, &c);
    tw[t] = C(c, s);
    f[t] = cexpi(-(c * a));
  }
  __syncthreads();
  const int nm = 2 * M + 3;
  const double inv = 1.0 / n_alpha;
  // f is even in alpha, so c_{-m} = c_m: m = 0..M+1 computed, mirrored
  for (int m = threadIdx.x; m <= M + 1; m += blockDim.x) {
    const int mm = m % n_alpha;
    cd acc = C(0.0);
    int idx = 0;
    for (int t = 0; t < n_alpha; ++t) {
      acc = fma(f[t], tw[idx], acc);
      idx += mm;
      if (idx >= n_alpha) idx -= n_alpha;
    }
    cd* dst = coef + ((size_t)p * g.N + j) * nm + (M + 1);
    dst[m] = inv * acc;
    dst[-m] = inv * acc;
  }
}

// F[w][p][q][3] for mode m = q - M: one CTA per (polar angle, mode, rhs)
__global__ void __launch_bounds__(128) ffgrid_mode_kernel(FieldGeom g, int M, cd k0, double omega, cd eps0,
                                                          int n_polar, const cd* __restrict__ coef,
                                                          const cd* __restrict__ x, int nrhs, cd* __restrict__ F) {
  const int p = blockIdx.x, q = blockIdx.y, w = blockIdx.z;
  const int nm = 2 * M + 3, n = 4 * g.N;
  double sth, cth;
  sincospi((p + 0.5) / n_polar, &sth, &cth);
  cd Jh[3] = {C(0.0), C(0.0), C(0.0)}, Mh[3] = {C(0.0), C(0.0), C(0.0)};
  const cd* xv = x + ((size_t)q * nrhs + w) * n;
  for (int j = threadIdx.x; j < g.N; j += blockDim.x) {
    const cd* cc = coef + ((size_t)p * g.N + j) * nm + q + 1;  // c_m at cc[0], c_{m-1} at cc[-1]
    const cd c0 = cc[0], cm = cc[-1], cp = cc[1];
    const cd Ic = 0.5 * (cp + cm);
    const cd Is = mul_i(0.5 * (cm - cp));                      // (c_{m+1} - c_{m-1})/(2i)
    const double wr = 6.283185307179586 * g.w[j] * g.r[j];
    const cd ph = wr * cexpi(-(k0 * (g.z[j] * cth)));
    const double rp = g.rp[j], zp = g.zp[j];
    const cd J1 = ph * xv[4 * j], J2 = ph * xv[4 * j + 1], M1 = ph * xv[4 * j + 2], M2 = ph * xv[4 * j + 3];
    Jh[0] += J1 * (rp * Ic) - J2 * Is;
    Jh[1] += J1 * (rp * Is) + J2 * Ic;
    Jh[2] += J1 * (zp * c0);
    Mh[0] += M1 * (rp * Ic) - M2 * Is;
    Mh[1] += M1 * (rp * Is) + M2 * Ic;
    Mh[2] += M1 * (zp * c0);
  }
  __shared__ cd red[6][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  cd v[6] = {Jh[0], Jh[1], Jh[2], Mh[0], Mh[1], Mh[2]};
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      v[a].x += __shfl_xor_sync(0xffffffffu, v[a].x, o);
      v[a].y += __shfl_xor_sync(0xffffffffu, v[a].y, o);
    }
    if (lane == 0) red[a][wid] = v[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cd t[6];
    for (int a = 0; a < 6; ++a) t[a] = red[a][0] + red[a][1] + red[a][2] + red[a][3];
    const double xh[3] = {sth, 0.0, cth};
    const cd xJ = xh[0] * t[0] + xh[2] * t[2];
    const cd pre = -(k0 * k0) / (C(0.0, omega) * eps0);
    const cd ik = mul_i(k0);
    cd cr[3];
    cr[0] = xh[1] * t[5] - xh[2] * t[4];
    cr[1] = xh[2] * t[3] - xh[0] * t[5];
    cr[2] = xh[0] * t[4] - xh[1] * t[3];
    const double inv4pi = 1.0 / (4.0 * 3.141592653589793);
    cd* dst = F + (((size_t)w * n_polar + p) * (2 * M + 1) + q) * 3;
    for (int a = 0; a < 3; ++a) dst[a] = inv4pi * (pre * (t[a] - xh[a] * xJ) + ik * cr[a]);
  }
}

// E[w][p][s][3] (Cartesian) = R_z(phi_s) sum_m e^{i m phi_s} F_m: one CTA per (polar angle, rhs)
__global__ void ffgrid_synth_kernel(int M, int n_polar, int n_azim, const cd* __restrict__ F, int nrhs,
                                    cd* __restrict__ E) {
  extern __shared__ __align__(16) char smem[];
  const int nq = 2 * M + 1;
  cd* Fs = (cd*)smem;          // [nq][3]
  cd* tw = Fs + 3 * nq;        // [n_azim] e^{2 pi i s / n_azim}
  const int p = blockIdx.x, w = blockIdx.y;
  const cd* src = F + ((size_t)w * n_polar + p) * nq * 3;
  for (int t = threadIdx.x; t < 3 * nq; t += blockDim.x) Fs[t] = src[t];
  for (int s = threadIdx.x; s < n_azim; s += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * s / n_azim, &sn, &cs);
    tw[s] = C(cs, sn);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n_azim; s += blockDim.x) {
    cd a[3] = {C(0.0), C(0.0), C(0.0)};
    int idx = (int)(((long long)(n_azim - (M % n_azim)) * s) % n_azim);  // (-M s) mod n_azim
    for (int q = 0; q < nq; ++q) {
      const cd e = tw[idx];
      a[0] = fma(Fs[3 * q], e, a[0]);
      a[1] = fma(Fs[3 * q + 1], e, a[1]);
      a[2] = fma(Fs[3 * q + 2], e, a[2]);
      idx += s;
      if (idx >= n_azim) idx -= n_azim;
    }
    const cd cphi = tw[s];  // (cos phi, sin phi)
    cd* dst = E + (((size_t)w * n_polar + p) * n_azim + s) * 3;
    dst[0] = cphi.x * a[0] - cphi.y * a[1];
    dst[1] = cphi.y * a[0] + cphi.x * a[1];
    dst[2] = a[2];
  }
}

void launch_far_field_grid(const FieldGeom& g, int M, cd k0, double omega, cd eps0, const cd* x, int nrhs,
                           int n_polar, int n_azim, int n_alpha, cd* coef, cd* F, cd* E, cudaStream_t s) {
  const int smem1 = 2 * n_alpha * (int)sizeof(cd);
  smem_optin(ffgrid_coef_kernel);
  ffgrid_coef_kernel<<<dim3(n_polar, g.N), 256, smem1, s>>>(g, M, k0, n_polar, n_alpha, coef);
  ffgrid_mode_kernel<<<dim3(n_polar, 2 * M + 1, nrhs), 128, 0, s>>>(g, M, k0, omega, eps0, n_polar, coef, x, nrhs,
                                                                    F);
  const int smem3 = (3 * (2 * M + 1) + n_azim) * (int)sizeof(cd);
  smem_optin(ffgrid_synth_kernel);
  ffgrid_synth_kernel<<<dim3(n_polar, nrhs), 256, smem3, s>>>(M, n_polar, n_azim, F, nrhs, E);
}

// Currents at refined nodes: xs[v][4s + a] = sum_k Lm[s][k] x[v][4 (node0[s] + k) + a]
// (v over modes x right-hand sides; the 16 nodes of sub-node s's panel);
// grid.y strides over the vectors.
__global__ void interp_currents_kernel(const cd* __restrict__ x, int n, int nsub, const int* __restrict__ node0,
                                       const double* __restrict__ Lm, long long nvec, cd* __restrict__ xs) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * nsub) return;
  const int s = idx >> 2, a = idx & 3;
  const double* L = Lm + (size_t)s * 16;
  for (long long v = blockIdx.y; v < nvec; v += gridDim.y) {
    const cd* xv = x + v * n + 4 * node0[s] + a;
    cd acc = C(0.0);
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(L[k], xv[4 * k], acc);
    xs[v * 4 * nsub + idx] = acc;
  }
}

void launch_interp_currents(const cd* x, int n, int nsub, const int* node0, const double* Lm, long long nvec, cd* xs,
                            cudaStream_t s) {
  const unsigned gy = (unsigned)(nvec < 65535 ? nvec : 65535);
  interp_currents_kernel<<<dim3((4 * nsub + 255) / 256, gy), 256, 0, s>>>(x, n, nsub, node0, Lm, nvec, xs);
}
