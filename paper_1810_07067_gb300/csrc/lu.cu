// Batched complex128 LU (right-looking, blocked by LU_NB columns) and solves.
//
// Per block column: (1) the panel is factored by one CTA per matrix with a
// warp-shuffle argmax for the pivot (largest |a|^2, lowest row on ties);
// (2) its row interchanges are applied to the other columns; (3) the block
// row of U is formed by a unit-lower triangular solve; (4) the trailing matrix
// is updated by a complex FP64 GEMM, batched over all matrices.
#include <cstdio>
#include <vector>
#include "lu.cuh"

// ---------------------------------------------------------------- panel
__device__ __forceinline__ void argmax_merge(double& v, int& idx, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
}

template <class T>
__global__ void __launch_bounds__(1024) panel_kernel(T* __restrict__ A, int n, int k0, int nbk,
                                                     int* __restrict__ piv, int* __restrict__ info) {
  const int b = blockIdx.x;
  T* M = A + (size_t)b * n * n;
  int* pv = piv + (size_t)b * n;
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  __shared__ T s_row[LU_NB];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, NT = blockDim.x;
  for (int jj = 0; jj < nbk; ++jj) {
    const int c = k0 + jj;
    T* col = M + (size_t)c * n;
    double best = -1.0;
    int bi = n;
    for (int r = c + tid; r < n; r += NT) argmax_merge(best, bi, norm2(col[r]), r);
    for (int o = 16; o > 0; o >>= 1) {
      double v2 = __shfl_xor_sync(0xffffffffu, best, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_merge(best, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
      best = (lane < (NT >> 5)) ? red_v[lane] : -1.0;
      bi = (lane < (NT >> 5)) ? red_i[lane] : n;
      for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(best, bi, v2, i2);
      }
      if (lane == 0) {
        s_p = (best > 0.0) ? bi : -1;
        pv[c] = (best > 0.0) ? bi : c;
        if (best <= 0.0 && info[b] == 0) info[b] = c + 1;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p >= 0) {
      if (p != c && tid < nbk) {
        T* cc = M + (size_t)(k0 + tid) * n;
        T t = cc[c]; cc[c] = cc[p]; cc[p] = t;
      }
      __syncthreads();
      if (tid < nbk) s_row[tid] = M[(size_t)(k0 + tid) * n + c];
      __syncthreads();
      const T inv = cone<T>() / s_row[jj];
      for (int r = c + 1 + tid; r < n; r += NT) {
        T l = col[r] * inv;
        col[r] = l;
        // the row's remaining panel entries in chunks of 8: loads batched, then updates
        for (int c0 = jj + 1; c0 < nbk; c0 += 8) {
          T v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + u < nbk) v[u] = M[(size_t)(k0 + c0 + u) * n + r];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + u < nbk) M[(size_t)(k0 + c0 + u) * n + r] = v[u] - l * s_row[c0 + u];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- swaps
template <class T>
__global__ void swap_kernel(T* __restrict__ A, int n, int k0, int nbk, const int* __restrict__ piv) {
  const int b = blockIdx.y;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int nother = n - nbk;
  if (c >= nother) return;
  if (c >= k0) c += nbk;  // skip the panel's own columns
  T* col = A + (size_t)b * n * n + (size_t)c * n;
  const int* pv = piv + (size_t)b * n;
  for (int k = k0; k < k0 + nbk; ++k) {
    int p = pv[k];
    if (p != k) { T t = col[k]; col[k] = col[p]; col[p] = t; }
  }
}

// ---------------------------------------------------------------- U12 = L11^{-1} A12
template <class T>
__global__ void trsm_kernel(T* __restrict__ A, int n, int k0, int nbk) {
  const int b = blockIdx.y;
  T* M = A + (size_t)b * n * n;
  __shared__ T L[LU_NB][LU_NB + 1];
  for (int t = threadIdx.x; t < nbk * nbk; t += blockDim.x) {
    int r = t % nbk, cc = t / nbk;
    L[r][cc] = M[(size_t)(k0 + cc) * n + k0 + r];
  }
  __syncthreads();
  int c = k0 + nbk + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  T* col = M + (size_t)c * n + k0;
  T x[LU_NB];
#pragma unroll
  for (int r = 0; r < LU_NB; ++r) x[r] = (r < nbk) ? col[r] : czero<T>();
#pragma unroll
  for (int k = 0; k < LU_NB; ++k) {
#pragma unroll
    for (int r = k + 1; r < LU_NB; ++r) x[r] = x[r] - L[r][k] * x[k];
  }
#pragma unroll
  for (int r = 0; r < LU_NB; ++r)
    if (r < nbk) col[r] = x[r];
}

// ---------------------------------------------------------------- trailing update
// C[i0.., j0..] -= A[i0.., k0..k0+nbk) * A[k0..k0+nbk), j0..], 64x64 tiles,
// 256 threads, each 4x4 outputs: rows tx + 16a, columns ty + 16b.
#define GT 64
template <class T>
__global__ void __launch_bounds__(256) gemm_update_kernel(T* __restrict__ A, int n, int k0, int nbk) {
  const int b = blockIdx.z;
  T* M = A + (size_t)b * n * n;
  const int start = k0 + nbk;
  const int i0 = start + blockIdx.x * GT, j0 = start + blockIdx.y * GT;
  __shared__ T As[LU_NB][GT];
  __shared__ T Bs[LU_NB][GT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int t = tid; t < nbk * GT; t += 256) {
    int r = t % GT, kk = t / GT;
    int gi = i0 + r;
    As[kk][r] = (gi < n) ? M[(size_t)(k0 + kk) * n + gi] : czero<T>();
    int kb = t % nbk, cj = t / nbk;  // B element (row k0+kb, column j0+cj)
    int gj = j0 + cj;
    Bs[kb][cj] = (gj < n) ? M[(size_t)gj * n + k0 + kb] : czero<T>();
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = czero<T>();
  for (int kk = 0; kk < nbk; ++kk) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
    for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][ty + 16 * c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int gj = j0 + ty + 16 * c;
    if (gj >= n) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int gi = i0 + tx + 16 * a;
      if (gi < n) {
        T* d = M + (size_t)gj * n + gi;
        *d = *d - acc[a][c];
      }
    }
  }
}

template <class T>
static void lu_factor_impl(T* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm) {
  cudaMemsetAsync(info, 0, sizeof(int) * batch, s);
  std::vector<cudaEvent_t> ev;
  int launches = 0;
  for (int k0 = 0; k0 < n; k0 += LU_NB) {
    int nbk = (n - k0 < LU_NB) ? n - k0 : LU_NB;
    panel_kernel<T><<<batch, 1024, 0, s>>>(A, n, k0, nbk, piv, info);
    ++launches;
    int nother = n - nbk;
    if (nother > 0) { swap_kernel<T><<<dim3((nother + 127) / 128, batch), 128, 0, s>>>(A, n, k0, nbk, piv); ++launches; }
    int rest = n - k0 - nbk;
    if (rest > 0) {
      trsm_kernel<T><<<dim3((rest + 127) / 128, batch), 128, 0, s>>>(A, n, k0, nbk);
      int t = (rest + GT - 1) / GT;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (tm) {
        cudaEventCreate(&e0); cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
      }
      gemm_update_kernel<T><<<dim3(t, t, batch), 256, 0, s>>>(A, n, k0, nbk);
      launches += 2;
      if (tm) {
        cudaEventRecord(e1, s);
        ev.push_back(e0); ev.push_back(e1);
        tm->gemm_flops += 8.0 * (double)rest * rest * nbk * batch;
        tm->gemm_launches += 1;
      }
    }
  }
  if (tm) {
    tm->launches += launches;
    if (!ev.empty()) cudaEventSynchronize(ev.back());
    for (size_t q = 0; q + 1 < ev.size(); q += 2) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
      tm->gemm_ms += ms;
      cudaEventDestroy(ev[q]); cudaEventDestroy(ev[q + 1]);
    }
  }
}

void lu_factor_batched(cd* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm) {
  lu_factor_impl<cd>(A, n, batch, piv, info, s, tm);
}

void lu_factor_batched_c64(cf* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm) {
  lu_factor_impl<cf>(A, n, batch, piv, info, s, tm);
}

// ---------------------------------------------------------------- solves
// Blocked forward/back substitution.  One CTA per (factor m, group of SG
// right-hand sides); a job is (rhs index, sign) with sign - meaning mode -m.
// The solution vectors are formed in place in x (each job owns its slot).
// Per block of SB rows: the SB x SB diagonal triangle is solved in shared
// memory, then the rows below (above, for U) are updated with the block column
// of the factor, which is read once per CTA.
#define SB 64
#define SG 8
__device__ __forceinline__ void job_of(int m, int M, int nrhs, int job, int* q, int* ridx, bool* neg) {
  *ridx = job % nrhs;
  *neg = job >= nrhs;
  *q = *neg ? (M - m) : (M + m);
}

template <class T> __device__ __forceinline__ T conv(cd a);
template <> __device__ __forceinline__ cd conv<cd>(cd a) { return a; }
template <> __device__ __forceinline__ cf conv<cf>(cd a) { return to_cf(a); }
__device__ __forceinline__ cd to_cd(cd a) { return a; }

// TF: factor type (cd, or cf for the mixed path's correction solves, which
// then run in FP32 arithmetic on FP64 storage).  PHYS: right-hand sides and
// solutions in physical unknowns (scaled by the sqrt weights here); otherwise
// both are already in the weighted space.
template <class TF, bool PHYS>
__global__ void __launch_bounds__(256) solve_blocked_kernel(const TF* __restrict__ LU, const int* __restrict__ piv,
                                                            int n, int M, const double* __restrict__ sw,
                                                            const cd* __restrict__ rhs, cd* __restrict__ x,
                                                            int nrhs) {
  __shared__ TF Ls[SB][SB + 1];
  __shared__ TF Xs[SB][SG];
  extern __shared__ int perm[];  // [n]: row interchanges composed into one permutation
  const int m = blockIdx.x;
  const int job0 = blockIdx.y * SG;
  const int njobs_all = (m == 0) ? nrhs : 2 * nrhs;
  if (job0 >= njobs_all) return;
  const int G = min(SG, njobs_all - job0);
  const TF* L = LU + (size_t)m * n * n;
  const int* pv = piv + (size_t)m * n;
  const int tid = threadIdx.x, T = blockDim.x;
  cd* X[SG];
  for (int g = 0; g < SG; ++g) {
    int q, ri; bool neg;
    job_of(m, M, nrhs, job0 + (g < G ? g : 0), &q, &ri, &neg);
    X[g] = x + ((size_t)q * nrhs + ri) * n;
  }
  // row interchanges (LAPACK order) composed into perm: (P b)[r] = b[perm[r]]
  for (int r = tid; r < n; r += T) perm[r] = r;
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < n; ++k) {
      int p = pv[k];
      if (p != k) { int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
    }
  }
  __syncthreads();
  // permuted, scaled (sqrt weights per node) and reflected right-hand sides
  for (int t = tid; t < G * n; t += T) {
    int g = t / n, r = t % n;
    int q, ri; bool neg;
    job_of(m, M, nrhs, job0 + g, &q, &ri, &neg);
    int src = perm[r];
    double sg = (neg && ((src & 3) == 0 || (src & 3) == 3)) ? -1.0 : 1.0;
    X[g][r] = ((PHYS ? sw[src >> 2] : 1.0) * sg) * rhs[((size_t)q * nrhs + ri) * n + src];
  }
  __syncthreads();
  // forward: L unit lower
  for (int kb = 0; kb < n; kb += SB) {
    const int bs = min(SB, n - kb);
    for (int t = tid; t < bs * bs; t += T) {
      int r = t % bs, c = t / bs;
      Ls[r][c] = L[(size_t)(kb + c) * n + kb + r];
    }
    for (int t = tid; t < bs * G; t += T) {
      int r = t % bs, g = t / bs;
      Xs[r][g] = conv<TF>(X[g][kb + r]);
    }
    __syncthreads();
    for (int c = 0; c < bs - 1; ++c) {
      for (int t = tid; t < (bs - 1 - c) * G; t += T) {
        int r = c + 1 + t % (bs - 1 - c), g = t / (bs - 1 - c);
        Xs[r][g] = Xs[r][g] - Ls[r][c] * Xs[c][g];
      }
      __syncthreads();
    }
    for (int t = tid; t < bs * G; t += T) {
      int r = t % bs, g = t / bs;
      X[g][kb + r] = to_cd(Xs[r][g]);
    }
    for (int r = kb + bs + tid; r < n; r += T) {
      TF acc[SG];
#pragma unroll
      for (int g = 0; g < SG; ++g) acc[g] = czero<TF>();
      for (int c = 0; c < bs; ++c) {
        TF l = L[(size_t)(kb + c) * n + r];
#pragma unroll
        for (int g = 0; g < SG; ++g) acc[g] = fma(l, Xs[c][g], acc[g]);
      }
      for (int g = 0; g < G; ++g) X[g][r] = X[g][r] - to_cd(acc[g]);
    }
    __syncthreads();
  }
  // backward: U upper, non-unit diagonal
  const int nblk = (n + SB - 1) / SB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int kb = bi * SB, bs = min(SB, n - kb);
    for (int t = tid; t < bs * bs; t += T) {
      int r = t % bs, c = t / bs;
      Ls[r][c] = L[(size_t)(kb + c) * n + kb + r];
    }
    for (int t = tid; t < bs * G; t += T) {
      int r = t % bs, g = t / bs;
      Xs[r][g] = conv<TF>(X[g][kb + r]);
    }
    __syncthreads();
    for (int c = bs - 1; c >= 0; --c) {
      if (tid < G) Xs[c][tid] = Xs[c][tid] / Ls[c][c];
      __syncthreads();
      for (int t = tid; t < c * G; t += T) {
        int r = t % c, g = t / c;
        Xs[r][g] = Xs[r][g] - Ls[r][c] * Xs[c][g];
      }
      __syncthreads();
    }
    for (int t = tid; t < bs * G; t += T) {
      int r = t % bs, g = t / bs;
      X[g][kb + r] = to_cd(Xs[r][g]);
    }
    for (int r = tid; r < kb; r += T) {
      TF acc[SG];
#pragma unroll
      for (int g = 0; g < SG; ++g) acc[g] = czero<TF>();
      for (int c = 0; c < bs; ++c) {
        TF u = L[(size_t)(kb + c) * n + r];
#pragma unroll
        for (int g = 0; g < SG; ++g) acc[g] = fma(u, Xs[c][g], acc[g]);
      }
      for (int g = 0; g < G; ++g) X[g][r] = X[g][r] - to_cd(acc[g]);
    }
    __syncthreads();
  }
  // back to physical unknowns (and reflection for -m)
  for (int t = tid; t < G * n; t += T) {
    int g = t / n, r = t % n;
    int q, ri; bool neg;
    job_of(m, M, nrhs, job0 + g, &q, &ri, &neg);
    double sg = (neg && ((r & 3) == 1 || (r & 3) == 2)) ? -1.0 : 1.0;
    X[g][r] = (sg / (PHYS ? sw[r >> 2] : 1.0)) * X[g][r];
  }
}

void lu_solve_modes(const cd* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x, int nrhs,
                    cudaStream_t s) {
  int groups = (2 * nrhs + SG - 1) / SG;
  int smem = n * (int)sizeof(int);
  cudaFuncSetAttribute(solve_blocked_kernel<cd, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  solve_blocked_kernel<cd, true><<<dim3(M + 1, groups), 256, smem, s>>>(LU, piv, n, M, sw, rhs, x, nrhs);
}

void lu_correction_solve_c64(const cf* LU, const int* piv, int n, int M, const cd* r, cd* d, int nrhs,
                             cudaStream_t s) {
  int groups = (2 * nrhs + SG - 1) / SG;
  int smem = n * (int)sizeof(int);
  cudaFuncSetAttribute(solve_blocked_kernel<cf, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  solve_blocked_kernel<cf, false><<<dim3(M + 1, groups), 256, smem, s>>>(LU, piv, n, M, nullptr, r, d, nrhs);
}
