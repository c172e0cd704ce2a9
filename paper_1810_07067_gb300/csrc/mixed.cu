// Mixed-precision solves (complex64 factors, FP64-accurate answers):
// the modes are factored in complex64 and every solve is refined with
// residuals of the complex128 L2-weighted matrices,
//   y_0 = LU32^{-1} b',  r_i = b' - A' y_i (FP64),  y_{i+1} = y_i + LU32^{-1} r_i,
// until ||r||_inf <= tol (||A'||_inf ||y||_inf + ||b'||_inf) for every mode and
// right-hand side.  Mode -m uses A'_{-m} = D_r A'_m D_c.
#include "mixed.cuh"

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// One pass over the complex128 matrices of the mixed path: the complex64
// copy the LU factors, the infinity norm of every matrix (for the stopping
// test) and, for the tensor-core residuals, every row's power-of-two scale
// (the smallest 2^e with max(|Re a|, |Im a|) over the row below 2^e / 2;
// 1 for empty rows and the padding rows n..npad-1).  32 rows x 8 column
// slices per block: a warp reads 32 consecutive rows of one column.
__device__ __forceinline__ double pow2_above_twice(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);             // mx = f 2^e, f in [1/2, 1)
  return ldexp(1.0, e + 1);  // mx / scale < 1/2
}

// The element loop keeps off the FP64 pipe (a small share of the SM on this
// part): the largest |Re a|, |Im a| is taken on the IEEE bit patterns (for
// non-negative doubles their order as unsigned integers is the numeric
// order), and the row sums of |a| run in FP32 per thread (the stopping test's
// norm needs no more), joined in FP64 across the block.
__global__ void __launch_bounds__(256) row_pass_kernel(const cd* __restrict__ A, int n, int npad, cf* __restrict__ A32,
                                                       double* __restrict__ normA, double* __restrict__ rowscale) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;  // slice 0..7
  const int i = blockIdx.x * 32 + lane;
  const cd* Mx = A + (size_t)b * n * n;
  cf* My = A32 ? A32 + (size_t)b * n * n : nullptr;  // null: norms only
  float s = 0.f;
  unsigned long long mxb = 0ull;  // bits of the largest |Re a|, |Im a|
  if (i < n) {
#pragma unroll 4
    for (int j = slice; j < n; j += 8) {
      const cd v = Mx[(size_t)j * n + i];
      const cf w = to_cf(v);
      if (My) My[(size_t)j * n + i] = w;
      const float fx = fabsf(w.x), fy = fabsf(w.y);
      const float hi = fmaxf(fx, fy), lo = fminf(fx, fy);
      const float q = (hi > 0.f) ? lo / hi : 0.f;
      s += hi * sqrtf(1.f + q * q);
      const unsigned long long bx = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull;
      const unsigned long long by = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull;
      mxb = max(mxb, max(bx, by));
    }
  }
  __shared__ double part[8][32];
  __shared__ unsigned long long pmax[8][32];
  part[slice][lane] = (double)s;
  pmax[slice][lane] = mxb;
  __syncthreads();
  if (slice == 0) {
    double t = 0.0;
    unsigned long long m2 = 0ull;
    for (int q = 0; q < 8; ++q) { t += part[q][lane]; m2 = max(m2, pmax[q][lane]); }
    if (rowscale && i < npad) rowscale[(size_t)b * npad + i] = pow2_above_twice(__longlong_as_double((long long)m2));
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) atomic_max_pos(normA + b, t);
  }
}

void mixed_prepare(const cd* A, int n, int batch, cf* A32, double* normA, double* rowscale, int npad, cudaStream_t s) {
  cudaMemsetAsync(normA, 0, sizeof(double) * batch, s);
  const int rows = rowscale ? npad : n;
  row_pass_kernel<<<dim3((rows + 31) / 32, batch), 256, 0, s>>>(A, n, rowscale ? npad : n, A32, normA, rowscale);
}

// Vector kernels: grid.y strides over the (mode, right-hand side) vectors, so
// any count fits the 65535 limit of gridDim.y.
static inline unsigned vec_grid(long long nvec) { return (unsigned)(nvec < 65535 ? nvec : 65535); }

__global__ void scale_kernel(const cd* __restrict__ b, cd* __restrict__ bw, const double* __restrict__ sw, int n,
                             long long nvec, double* __restrict__ bnorm) {
  for (long long v = blockIdx.y; v < nvec; v += gridDim.y) {
    double mx = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
      cd val = sw[r >> 2] * b[v * n + r];
      bw[v * n + r] = val;
      mx = fmax(mx, cabs(val));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomic_max_pos(bnorm + v, mx);
  }
}

void mixed_scale(const cd* b, cd* bw, const double* sw, int n, long long nvec, double* bnorm, cudaStream_t s) {
  cudaMemsetAsync(bnorm, 0, sizeof(double) * nvec, s);
  scale_kernel<<<dim3((n + 255) / 256, vec_grid(nvec)), 256, 0, s>>>(b, bw, sw, n, nvec, bnorm);
}

__global__ void update_kernel(cd* __restrict__ y, const cd* __restrict__ d, int n, long long nvec, bool first,
                              double* __restrict__ ynorm) {
  for (long long v = blockIdx.y; v < nvec; v += gridDim.y) {
    double mx = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
      cd val = first ? d[v * n + r] : y[v * n + r] + d[v * n + r];
      y[v * n + r] = val;
      mx = fmax(mx, cabs(val));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomic_max_pos(ynorm + v, mx);
  }
}

void mixed_update(cd* y, const cd* d, int n, long long nvec, bool first, double* ynorm, cudaStream_t s) {
  cudaMemsetAsync(ynorm, 0, sizeof(double) * nvec, s);
  update_kernel<<<dim3((n + 255) / 256, vec_grid(nvec)), 256, 0, s>>>(y, d, n, nvec, first, ynorm);
}

__global__ void unscale_kernel(const cd* __restrict__ y, cd* __restrict__ x, const double* __restrict__ sw, int n,
                               long long nvec) {
  for (long long v = blockIdx.y; v < nvec; v += gridDim.y)
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
      x[v * n + r] = (1.0 / sw[r >> 2]) * y[v * n + r];
}

void mixed_unscale(const cd* y, cd* x, const double* sw, int n, long long nvec, cudaStream_t s) {
  unscale_kernel<<<dim3((n + 255) / 256, vec_grid(nvec)), 256, 0, s>>>(y, x, sw, n, nvec);
}

// Residual GEMM: Z = A'_m [y_{+m}, D_c y_{-m}] for a 64-row x 32-job tile,
// then r = b' - Z (and D_r Z for -m).  256 threads, 8 outputs each.
#define RT 64
#define RJ 32
#define RK 32
__global__ void __launch_bounds__(256) residual_kernel(const cd* __restrict__ A, int n, int M,
                                                       const cd* __restrict__ bw, const cd* __restrict__ y,
                                                       cd* __restrict__ r, int nrhs, double* __restrict__ rnorm) {
  const int m = blockIdx.y;
  const int i0 = blockIdx.x * RT, j0 = blockIdx.z * RJ;
  const int njobs = 2 * nrhs;
  const cd* Am = A + (size_t)m * n * n;
  __shared__ cd As[RK][RT];
  __shared__ cd Ys[RK][RJ];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  cd acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) { acc[a][0] = C(0.0); acc[a][1] = C(0.0); }
  for (int k0 = 0; k0 < n; k0 += RK) {
    for (int t = tid; t < RK * RT; t += 256) {
      int rr = t % RT, kk = t / RT;
      int gi = i0 + rr, gk = k0 + kk;
      As[kk][rr] = (gi < n && gk < n) ? Am[(size_t)gk * n + gi] : C(0.0);
    }
    for (int t = tid; t < RK * RJ; t += 256) {
      int kk = t % RK, jj = t / RK;
      int job = j0 + jj, gk = k0 + kk;
      cd v = C(0.0);
      if (job < njobs && gk < n && !(m == 0 && job >= nrhs)) {
        bool neg = job >= nrhs;
        int ridx = neg ? job - nrhs : job;
        int q = neg ? M - m : M + m;
        v = y[((size_t)q * nrhs + ridx) * n + gk];
        if (neg && ((gk & 3) == 1 || (gk & 3) == 2)) v = -v;   // D_c
      }
      Ys[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < RK; ++kk) {
      cd y0 = Ys[kk][ty], y1 = Ys[kk][ty + 16];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        cd av = As[kk][tx + 16 * a];
        acc[a][0] = fma(av, y0, acc[a][0]);
        acc[a][1] = fma(av, y1, acc[a][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    int job = j0 + ty + 16 * c;
    if (job >= njobs || (m == 0 && job >= nrhs)) continue;
    bool neg = job >= nrhs;
    int ridx = neg ? job - nrhs : job;
    int q = neg ? M - m : M + m;
    double mx = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int gi = i0 + tx + 16 * a;
      if (gi >= n) continue;
      cd z = acc[a][c];
      if (neg && ((gi & 3) == 0 || (gi & 3) == 3)) z = -z;    // D_r
      size_t idx = ((size_t)q * nrhs + ridx) * n + gi;
      cd val = bw[idx] - z;
      r[idx] = val;
      mx = fmax(mx, cabs(val));
    }
    atomic_max_pos(rnorm + (size_t)q * nrhs + ridx, mx);
  }
}

void mixed_residual(const cd* A, int n, int M, const cd* bw, const cd* y, cd* r, int nrhs, double* rnorm,
                    cudaStream_t s) {
  cudaMemsetAsync(rnorm, 0, sizeof(double) * (2 * M + 1) * nrhs, s);
  dim3 grid((n + RT - 1) / RT, M + 1, (2 * nrhs + RJ - 1) / RJ);
  residual_kernel<<<grid, 256, 0, s>>>(A, n, M, bw, y, r, nrhs, rnorm);
}
