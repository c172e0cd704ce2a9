// Condition estimate of every mode's factored system (the paper's LAPACK
// ZGESVX runs of Section 6 report condition numbers of the mode-0 systems).
//
// kappa_inf(A') = ||A'||_inf ||A'^{-1}||_inf for the L2-weighted matrix of each
// mode, with ||A'^{-1}||_inf = ||A'^{-H}||_1 estimated by Hager's method as
// refined by Higham (the iteration of LAPACK's xLACN2): with B = A'^{-H},
//   x = e / n; y = B x; est = ||y||_1; xi = sign(y); z = B^H xi; j = argmax |z|;
//   repeat (at most 5 times): x = e_j; y = B x; stop unless ||y||_1 > est;
//     est = ||y||_1; xi = sign(y); z = B^H xi; stop if max |z| is at j again;
//   finally est = max(est, 2 ||B x_alt||_1 / (3n)), x_alt_i = (-1)^i (1 + i/(n-1)).
// B x is a solve with A'^H = U^H L^H P and B^H xi a solve with A' = P^T L U,
// both with the LU factors of the build (P A' = L U).  One CTA per mode; the
// vectors live in global scratch.  The estimate is a lower bound of
// ||A'^{-1}||_inf, in practice within a small factor of it.
#include <cuda_runtime.h>
#include "cplx.cuh"

#define COND_THREADS 1024

template <class T> __device__ __forceinline__ cd ld(const T* p);
template <> __device__ __forceinline__ cd ld<cd>(const cd* p) { return *p; }
template <> __device__ __forceinline__ cd ld<cf>(const cf* p) { const cf v = *p; return cd{(double)v.x, (double)v.y}; }

__device__ __forceinline__ cd conjd(cd a) { return cd{a.x, -a.y}; }

// Sum of a per-thread complex value over the CTA; every thread gets the total.
__device__ cd block_sum(cd v, cd* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  cd t{0.0, 0.0};
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = t + red[q];
  return t;
}

// x <- A'^{-1} x with P A' = L U
template <class T>
__device__ void solve_a(const T* __restrict__ LU, const int* __restrict__ piv, int n, cd* x) {
  if (threadIdx.x == 0)
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) { cd t = x[k]; x[k] = x[p]; x[p] = t; }
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {  // L: unit lower, by columns
    const cd xk = x[k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) x[i] = x[i] - ld(LU + (size_t)k * n + i) * xk;
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {  // U: upper, by columns
    if (threadIdx.x == 0) x[k] = x[k] / ld(LU + (size_t)k * n + k);
    __syncthreads();
    const cd xk = x[k];
    for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = x[i] - ld(LU + (size_t)k * n + i) * xk;
    __syncthreads();
  }
}

// x <- A'^{-H} x: A'^H = U^H L^H P, so solve U^H w = x, L^H v = w, x = P^T v
template <class T>
__device__ void solve_ah(const T* __restrict__ LU, const int* __restrict__ piv, int n, cd* x, cd* red) {
  for (int i = 0; i < n; ++i) {  // U^H is lower: w_i = (x_i - sum_{k<i} conj(U_ki) w_k) / conj(U_ii)
    cd s{0.0, 0.0};
    for (int k = threadIdx.x; k < i; k += blockDim.x) s = s + conjd(ld(LU + (size_t)i * n + k)) * x[k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) x[i] = (x[i] - s) / conjd(ld(LU + (size_t)i * n + i));
    __syncthreads();
  }
  for (int i = n - 1; i >= 0; --i) {  // L^H is unit upper: v_i = w_i - sum_{k>i} conj(L_ki) v_k
    cd s{0.0, 0.0};
    for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) s = s + conjd(ld(LU + (size_t)i * n + k)) * x[k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) x[i] = x[i] - s;
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = n - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k) { cd t = x[k]; x[k] = x[p]; x[p] = t; }
    }
  __syncthreads();
}

__device__ double block_max_abs(const cd* x, int n, int* arg, double* redd, int* redi) {
  double best = -1.0;
  int bi = n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = cabs(x[i]);
    if (a > best || (a == best && i < bi)) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double b2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { redd[w] = best; redi[w] = bi; }
  __syncthreads();
  best = -1.0; bi = n;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
    if (redd[q] > best || (redd[q] == best && redi[q] < bi)) { best = redd[q]; bi = redi[q]; }
  *arg = bi;
  return best;
}

__device__ double block_norm1(const cd* x, int n, cd* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += cabs(x[i]);
  return block_sum(cd{s, 0.0}, red).x;
}

template <class T>
__global__ void __launch_bounds__(COND_THREADS) cond_kernel(const T* __restrict__ LU, const int* __restrict__ piv,
                                                           int n, const double* __restrict__ normA,
                                                           cd* __restrict__ work, double* __restrict__ kappa) {
  const int m = blockIdx.x;
  const T* F = LU + (size_t)m * n * n;
  const int* pv = piv + (size_t)m * n;
  cd* x = work + (size_t)m * n;
  __shared__ cd red[COND_THREADS / 32];
  __shared__ double redd[COND_THREADS / 32];
  __shared__ int redi[COND_THREADS / 32];
  // B = A'^{-H}: B x by solve_ah, B^H x by solve_a
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = cd{1.0 / n, 0.0};
  __syncthreads();
  solve_ah(F, pv, n, x, red);
  double est = block_norm1(x, n, red);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {  // xi = sign(y)
    const double a = cabs(x[i]);
    x[i] = a > 0.0 ? x[i] / a : cd{1.0, 0.0};
  }
  __syncthreads();
  solve_a(F, pv, n, x);
  int j = 0;
  block_max_abs(x, n, &j, redd, redi);
  for (int it = 0; it < 5; ++it) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = cd{i == j ? 1.0 : 0.0, 0.0};
    __syncthreads();
    solve_ah(F, pv, n, x, red);
    const double e2 = block_norm1(x, n, red);
    if (!(e2 > est)) break;
    est = e2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double a = cabs(x[i]);
      x[i] = a > 0.0 ? x[i] / a : cd{1.0, 0.0};
    }
    __syncthreads();
    solve_a(F, pv, n, x);
    int j2 = 0;
    const double zmax = block_max_abs(x, n, &j2, redd, redi);
    if (cabs(x[j]) >= zmax) break;  // the maximum is where it was
    j = j2;
    __syncthreads();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    x[i] = cd{((i & 1) ? -1.0 : 1.0) * (1.0 + (n > 1 ? (double)i / (n - 1) : 0.0)), 0.0};
  __syncthreads();
  solve_ah(F, pv, n, x, red);
  const double alt = 2.0 * block_norm1(x, n, red) / (3.0 * n);
  if (threadIdx.x == 0) kappa[m] = normA[m] * fmax(est, alt);
}

void launch_cond_estimate(const void* LU, bool c64, const int* piv, int n, int modes, const double* normA, cd* work,
                          double* kappa, cudaStream_t s) {
  if (c64) cond_kernel<cf><<<modes, COND_THREADS, 0, s>>>((const cf*)LU, piv, n, normA, work, kappa);
  else cond_kernel<cd><<<modes, COND_THREADS, 0, s>>>((const cd*)LU, piv, n, normA, work, kappa);
}
