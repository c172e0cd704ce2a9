// Incident data and far fields (Section 6).
#include "fields.cuh"

// One CTA per (node, wave): samples of the tangential traces on the node's
// ring at n_theta azimuths, then their Fourier coefficients for m = -M..M.
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
    // E components in (e_r, e_theta, e_z)
    double Er = e[0] * ct + e[1] * st, Et = -e[0] * st + e[1] * ct, Ez = e[2];
    double Hr = hx * ct + hy * st, Ht = -hx * st + hy * ct, Hz = hz;
    // n x v = v_theta t - v_t e_theta
    smp[4 * t + 0] = Et * ph;
    smp[4 * t + 1] = -(rp * Er + zp * Ez) * ph;
    smp[4 * t + 2] = Ht * (hf * ph);
    smp[4 * t + 3] = -(rp * Hr + zp * Hz) * (hf * ph);
  }
  __syncthreads();
  const int n = 4 * g.N;
  const double inv = 1.0 / n_theta;
  // one (mode, component) per item: the DFT sum over the ring samples
  for (int item = threadIdx.x; item < 4 * (2 * M + 1); item += blockDim.x) {
    const int mq = item >> 2, a = item & 3;
    const int m = mq - M;
    const int mm = ((m % n_theta) + n_theta) % n_theta;
    cd acc = C(0.0);
    int idx = 0;
    for (int t = 0; t < n_theta; ++t) {
      acc = fma(smp[4 * t + a], tw[idx], acc);
      idx += mm;
      if (idx >= n_theta) idx -= n_theta;
    }
    rhs[((size_t)mq * nrhs + w) * n + 4 * i + a] = (a < 2 ? sE : sH) * (inv * acc);
  }
}

void launch_rhs_planewave(const FieldGeom& g, int M, cd k0, double omega, cd mu0, cd sE, cd sH,
                          const double* dirs_dev, const double* pols_dev, int nrhs, int n_theta, cd* rhs,
                          cudaStream_t s) {
  int smem = n_theta * 5 * (int)sizeof(cd);
  cudaFuncSetAttribute(rhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
