// Batched complex128 LU (right-looking, blocked by LU_NB columns) and solves.
//
// Per block column: (1) the panel is factored by one CTA per matrix with a
// warp-shuffle argmax for the pivot (largest |a|^2, lowest row on ties);
// (2) its row interchanges are applied to the other columns; (3) the block
// row of U is formed by a unit-lower triangular solve; (4) the trailing matrix
// is updated by a complex FP64 GEMM, batched over all matrices.
#include <cstdio>
#include <type_traits>
#include <vector>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include "lu.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

// ---------------------------------------------------------------- panel
// Pivot measure: |a|^2 in FP64 for complex128; |Re a| + |Im a| in FP32 for
// complex64 (LAPACK's complex pivot measure; GB300's FP64 pipe is too slow to
// sit on the panel's critical path).  Largest measure, lowest row on ties.
template <class T> struct Pivot;
template <> struct Pivot<cd> {
  using V = double;
  __device__ static V measure(cd a) { return norm2(a); }
};
template <> struct Pivot<cf> {
  using V = float;
  __device__ static V measure(cf a) { return fabsf(a.x) + fabsf(a.y); }
};

template <class V>
__device__ __forceinline__ void argmax_merge(V& v, int& idx, V v2, int i2) {
  if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
}

template <class T>
__global__ void __launch_bounds__(1024) panel_kernel(T* __restrict__ A, int n, int k0, int nbk,
                                                     int* __restrict__ piv, int* __restrict__ info) {
  const int b = blockIdx.x;
  T* M = A + (size_t)b * n * n;
  int* pv = piv + (size_t)b * n;
  using V = typename Pivot<T>::V;
  __shared__ V red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  __shared__ T s_row[LU_NB];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, NT = blockDim.x;
  for (int jj = 0; jj < nbk; ++jj) {
    const int c = k0 + jj;
    T* col = M + (size_t)c * n;
    V best = V(-1);
    int bi = n;
    for (int r = c + tid; r < n; r += NT) argmax_merge(best, bi, Pivot<T>::measure(col[r]), r);
    for (int o = 16; o > 0; o >>= 1) {
      V v2 = __shfl_xor_sync(0xffffffffu, best, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_merge(best, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
      best = (lane < (NT >> 5)) ? red_v[lane] : V(-1);
      bi = (lane < (NT >> 5)) ? red_i[lane] : n;
      for (int o = 16; o > 0; o >>= 1) {
        V v2 = __shfl_xor_sync(0xffffffffu, best, o);
        int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(best, bi, v2, i2);
      }
      if (lane == 0) {
        s_p = (best > V(0)) ? bi : -1;
        pv[c] = (best > V(0)) ? bi : c;
        if (best <= V(0) && info[b] == 0) info[b] = c + 1;
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

// ---------------------------------------------------------------- cluster panel
// The panel (rows k0..n-1, nbk columns) held in the shared memory of a
// cluster of C CTAs: CTA q owns rows k0 + q R .. k0 + (q+1) R - 1 as a
// column-major slice [nbk][R].  Per column: local argmax, candidates written
// into every CTA's shared memory through the cluster's distributed shared
// memory, cluster barrier; the pivot row's owner broadcasts it (and the
// displaced row is sent to the pivot's owner), cluster barrier; then the
// interchange and the rank-1 update of the owned rows.  Same pivot rule as
// panel_kernel (largest |a|^2, lowest row on ties).
#define PANEL_SMEM_MAX (200 * 1024)
#define PANEL_THREADS 512

template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) panel_cluster_kernel(T* __restrict__ A, int n, int k0, int nbk,
                                                                      int R, int* __restrict__ piv,
                                                                      int* __restrict__ info) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int b = blockIdx.y;
  T* M = A + (size_t)b * n * n;
  int* pv = piv + (size_t)b * n;
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T* a = (T*)panel_smem;  // [nbk][R]
  using V = typename Pivot<T>::V;
  __shared__ V cand_v[8];
  __shared__ int cand_i[8];
  __shared__ T s_row[LU_NB], s_rowc[LU_NB];
  __shared__ V red_v[PANEL_THREADS / 32];
  __shared__ int red_i[PANEL_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int row0 = k0 + q * R;
  const int nr = max(0, min(R, n - row0));  // rows owned by this CTA
  for (int t = tid; t < nbk * nr; t += PANEL_THREADS) {
    int r = t % nr, j = t / nr;
    a[j * R + r] = M[(size_t)(k0 + j) * n + row0 + r];
  }
  __syncthreads();
  for (int jj = 0; jj < nbk; ++jj) {
    const int c = k0 + jj;
    const T* aj = a + jj * R;
    V best = V(-1);
    int bi = n;
    for (int r = max(0, c - row0) + tid; r < nr; r += PANEL_THREADS)
      argmax_merge(best, bi, Pivot<T>::measure(aj[r]), row0 + r);
    for (int o = 16; o > 0; o >>= 1) {
      V v2 = __shfl_xor_sync(0xffffffffu, best, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_merge(best, bi, v2, i2);
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
      best = (lane < PANEL_THREADS / 32) ? red_v[lane] : V(-1);
      bi = (lane < PANEL_THREADS / 32) ? red_i[lane] : n;
      for (int o = 16; o > 0; o >>= 1) {
        V v2 = __shfl_xor_sync(0xffffffffu, best, o);
        int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(best, bi, v2, i2);
      }
      if (lane < C) {  // this CTA's candidate into slot q of every CTA
        cl.map_shared_rank(cand_v, lane)[q] = best;
        cl.map_shared_rank(cand_i, lane)[q] = bi;
      }
    }
    cl.sync();
    best = V(-1);
    bi = n;
    for (int u = 0; u < C; ++u) argmax_merge(best, bi, cand_v[u], cand_i[u]);
    const int p = (best > V(0)) ? bi : -1;
    if (q == 0 && tid == 0) {
      pv[c] = (p >= 0) ? p : c;
      if (p < 0 && info[b] == 0) info[b] = c + 1;
    }
    const int qp = (p >= 0) ? (p - k0) / R : -1, qc = (c - k0) / R;
    if (p >= 0) {
      if (q == qp && tid < nbk * C) {
        int j = tid % nbk, u = tid / nbk;
        cl.map_shared_rank(s_row, u)[j] = a[j * R + p - row0];
      }
      if (q == qc && p != c && tid < nbk) cl.map_shared_rank(s_rowc, qp)[tid] = a[tid * R + c - row0];
    }
    cl.sync();
    if (p >= 0) {
      if (q == qc && tid < nbk) a[tid * R + c - row0] = s_row[tid];
      if (q == qp && p != c && tid < nbk) a[tid * R + p - row0] = s_rowc[tid];
      __syncthreads();
      const T inv = cone<T>() / s_row[jj];
      for (int r = max(0, c + 1 - row0) + tid; r < nr; r += PANEL_THREADS) {
        T l = a[jj * R + r] * inv;
        a[jj * R + r] = l;
        for (int j = jj + 1; j < nbk; ++j) a[j * R + r] = a[j * R + r] - l * s_row[j];
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < nbk * nr; t += PANEL_THREADS) {
    int r = t % nr, j = t / nr;
    M[(size_t)(k0 + j) * n + row0 + r] = a[j * R + r];
  }
  cl.sync();  // no CTA leaves while a peer could still address its shared memory
}

// Cluster size: the smallest of 1, 2, 4, 8 whose row slices fit PANEL_SMEM_MAX.
// Returns false (nothing launched) when none fits or no such cluster can be
// resident; the caller then uses panel_kernel.
template <class T>
static bool launch_panel_cluster(T* A, int n, int k0, int nbk, int batch, int* piv, int* info, cudaStream_t s) {
  const int rows = n - k0;
  int C = 1;
  while (C < 8 && (size_t)LU_NB * ((rows + C - 1) / C) * sizeof(T) > PANEL_SMEM_MAX) C *= 2;
  const int R = (rows + C - 1) / C;
  const size_t smem = (size_t)LU_NB * R * sizeof(T);
  if (smem > PANEL_SMEM_MAX) return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM_MAX) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, batch);
  cfg.blockDim = dim3(PANEL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, panel_cluster_kernel<T>, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  if (cudaLaunchKernelEx(&cfg, panel_cluster_kernel<T>, A, n, k0, nbk, R, piv, info) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// ---------------------------------------------------------------- swaps
// The nbk interchanges of a block column compose to a permutation of at most
// 2 nbk rows: the block's own rows (slots 0..nbk-1) and the distinct targets
// below it (slot nbk + lane of the first interchange naming it).  One warp
// forms it per CTA; each warp then moves the affected entries of its columns
// (all loads before all stores).
#define SWAP_COLS 64
template <class T>
__global__ void __launch_bounds__(256) swap_kernel(T* __restrict__ A, int n, int k0, int nbk,
                                                   const int* __restrict__ piv) {
  const int b = blockIdx.y;
  __shared__ int pos[2 * LU_NB], src[2 * LU_NB], slot[LU_NB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kend = k0 + nbk;
  if (warp == 0) {
    const int p = (lane < nbk) ? piv[(size_t)b * n + k0 + lane] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, p);
    const bool below = p >= kend;
    const bool first = below && (__ffs(same) - 1 == lane);
    const int sp = (lane >= nbk) ? 0 : (below ? LU_NB + __ffs(same) - 1 : p - k0);
    pos[lane] = (lane < nbk) ? k0 + lane : -1;
    src[lane] = pos[lane];
    pos[LU_NB + lane] = first ? p : -1;
    src[LU_NB + lane] = first ? p : -1;
    slot[lane] = sp;
    __syncwarp();
    if (lane == 0)
      for (int k = 0; k < nbk; ++k) {
        const int s2 = slot[k];
        if (s2 != k) { int t = src[k]; src[k] = src[s2]; src[s2] = t; }
      }
  }
  __syncthreads();
  const int d0 = pos[lane], d1 = pos[lane + 32], s0 = src[lane], s1 = src[lane + 32];
  for (int cc = warp; cc < SWAP_COLS; cc += 8) {
    int c = blockIdx.x * SWAP_COLS + cc;
    if (c >= n - nbk) break;  // whole warp
    if (c >= k0) c += nbk;     // skip the panel's own columns
    T* col = A + (size_t)b * n * n + (size_t)c * n;
    T v0 = czero<T>(), v1 = czero<T>();
    if (d0 >= 0 && d0 != s0) v0 = col[s0];
    if (d1 >= 0 && d1 != s1) v1 = col[s1];
    __syncwarp();
    if (d0 >= 0 && d0 != s0) col[d0] = v0;
    if (d1 >= 0 && d1 != s1) col[d1] = v1;
    __syncwarp();
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

// ---------------------------------------------------------------- tensor-core trailing update
// Complex64 trailing update C -= L U on tcgen05: every FP32 operand is split
// exactly into three BF16 pieces (x = hi + mid + lo, 24 bits), and the six
// piece products whose sum carries FP32 precision (hh, hm, mh, hl, mm, lh) are
// accumulated in FP32 tensor memory (-L_im U_im via the MMA's A-negation).
// The hi*hi products and the five smaller corrections go to separate
// accumulators (Re and Im each, four in all) that are added in registers:
// sharing one accumulator loses about two bits to the tensor core's
// accumulation, which measured 4x the error of a plain FP32 update, while the
// split form measured half of it.  One CTA per 128 x 64 output tile of one
// matrix; 128 threads; operands are re-laid out into the MMA's K-major
// no-swizzle core-matrix format in shared memory.
#define TCU_M 128
#define TCU_N 64
#define TCU_ATILE (TCU_M * LU_NB)  // bf16 elements per piece tile of L (128 rows x 32 k)
#define TCU_BTILE (TCU_N * LU_NB)  // of U (64 columns x 32 k)
#define TCU_SMEM (6 * (TCU_ATILE + TCU_BTILE) * 2)

__device__ __forceinline__ int tcu_off(int r, int k) {  // 4 core matrices along k
  return ((r >> 3) * (LU_NB / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16* p) {
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  float r1 = x - __bfloat162float(h);
  __nv_bfloat16 m = __float2bfloat16_rn(r1);
  float r2 = r1 - __bfloat162float(m);
  p[0] = h; p[1] = m; p[2] = __float2bfloat16_rn(r2);
}

// Per step, the L panel (rows start.., 32 columns) and the U panel (32 rows,
// columns start..) are split once into their BF16 pieces, stored tile by tile
// in exactly the shared-memory image the MMAs read: per matrix, ceil(n/128)
// L tiles of [6 pieces][128 x 32], then ceil(n/64) U tiles of [6][64 x 32].
__host__ __device__ inline size_t tcu_ws_matrix_elems(int n) {
  return (size_t)((n + TCU_M - 1) / TCU_M) * 6 * TCU_ATILE + (size_t)((n + TCU_N - 1) / TCU_N) * 6 * TCU_BTILE;
}

size_t lu_c64_workspace_bytes(int n, int batch) { return tcu_ws_matrix_elems(n) * (size_t)batch * 2; }

__global__ void __launch_bounds__(256) tcu_split_kernel(const cf* __restrict__ A, int n, int k0, int nbk, int nL,
                                                       __nv_bfloat16* __restrict__ ws) {
  const int b = blockIdx.y;
  const cf* M = A + (size_t)b * n * n;
  const int start = k0 + nbk;
  __nv_bfloat16* W = ws + (size_t)b * tcu_ws_matrix_elems(n);
  __nv_bfloat16 pr[3], pi[3];
  if ((int)blockIdx.x < nL) {
    const int r0 = start + blockIdx.x * TCU_M;
    __nv_bfloat16* dst = W + (size_t)blockIdx.x * 6 * TCU_ATILE;
    for (int t = threadIdx.x; t < TCU_M * LU_NB; t += 256) {
      int r = t % TCU_M, k = t / TCU_M;
      cf v = (r0 + r < n && k < nbk) ? M[(size_t)(k0 + k) * n + r0 + r] : CF(0.f);
      split3(v.x, pr); split3(v.y, pi);
      int off = tcu_off(r, k);
#pragma unroll
      for (int q = 0; q < 3; ++q) { dst[q * TCU_ATILE + off] = pr[q]; dst[(3 + q) * TCU_ATILE + off] = pi[q]; }
    }
  } else {
    const int y = blockIdx.x - nL, c0 = start + y * TCU_N;
    __nv_bfloat16* dst = W + (size_t)((n + TCU_M - 1) / TCU_M) * 6 * TCU_ATILE + (size_t)y * 6 * TCU_BTILE;
    for (int t = threadIdx.x; t < TCU_N * LU_NB; t += 256) {
      int k = t % LU_NB, j = t / LU_NB;
      cf v = (c0 + j < n && k < nbk) ? M[(size_t)(c0 + j) * n + k0 + k] : CF(0.f);
      split3(v.x, pr); split3(v.y, pi);
      int off = tcu_off(j, k);
#pragma unroll
      for (int q = 0; q < 3; ++q) { dst[q * TCU_BTILE + off] = pr[q]; dst[(3 + q) * TCU_BTILE + off] = pi[q]; }
    }
  }
}

// Launched with TCU_SMEM_LAUNCH bytes of dynamic shared memory so that at
// most two CTAs share an SM (each holds 256 TMEM columns of the 512).
#define TCU_SMEM_LAUNCH (100 * 1024)

__global__ void __launch_bounds__(128) gemm_update_tc_kernel(cf* __restrict__ A, int n, int k0, int nbk,
                                                            const __nv_bfloat16* __restrict__ ws,
                                                            int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __nv_bfloat16* As = (__nv_bfloat16*)smem;
  __nv_bfloat16* Bs = As + 6 * TCU_ATILE;
  __shared__ __align__(8) uint64_t mbar_load, mbar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  const int b = blockIdx.z;
  cf* M = A + (size_t)b * n * n;
  const int start = k0 + nbk;
  const int i0 = start + blockIdx.x * TCU_M, j0 = start + blockIdx.y * TCU_N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 4 * TCU_N);
  if (tid == 0) {
    s_ok = 1;
    tc::mbar_init(&mbar_load, 1);
    tc::mbar_init(&mbar_mma, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  // accumulator columns: [0,N) hh Re, [N,2N) hh Im, [2N,3N) corrections Re, [3N,4N) corrections Im
  if (tid == 0) {
    const __nv_bfloat16* W = ws + (size_t)b * tcu_ws_matrix_elems(n);
    const __nv_bfloat16* Lsrc = W + (size_t)blockIdx.x * 6 * TCU_ATILE;
    const __nv_bfloat16* Usrc =
        W + (size_t)((n + TCU_M - 1) / TCU_M) * 6 * TCU_ATILE + (size_t)blockIdx.y * 6 * TCU_BTILE;
    tc::mbar_expect_tx(&mbar_load, TCU_SMEM);
    tc::bulk_g2s(As, Lsrc, 6 * TCU_ATILE * 2, &mbar_load);
    tc::bulk_g2s(Bs, Usrc, 6 * TCU_BTILE * 2, &mbar_load);
    if (tc::mbar_wait(&mbar_load, 0)) {
      tc::fence_after();
      const uint32_t id_pos = tc::idesc_bf16_f32(TCU_M, TCU_N, false);
      const uint32_t id_neg = tc::idesc_bf16_f32(TCU_M, TCU_N, true);
      const uint64_t a0 = tc::desc_noswizzle(tc::smem_u32(As), 128, (LU_NB / 8) * 128);
      const uint64_t b0 = tc::desc_noswizzle(tc::smem_u32(Bs), 128, (LU_NB / 8) * 128);
      const uint64_t at = (uint64_t)(TCU_ATILE * 2 / 16), bt = (uint64_t)(TCU_BTILE * 2 / 16);  // 16-byte units
      const int qa_[6] = {0, 0, 1, 0, 1, 2}, qb_[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int ks = 0; ks < LU_NB / 16; ++ks) {
        const uint64_t kof = (uint64_t)(ks * 256 / 16);  // two core matrices along k
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          const uint64_t are = a0 + qa_[u] * at + kof, aim = a0 + (3 + qa_[u]) * at + kof;
          const uint64_t bre = b0 + qb_[u] * bt + kof, bim = b0 + (3 + qb_[u]) * bt + kof;
          const uint32_t dre = tmem + (u == 0 ? 0 : 2 * TCU_N), dim = tmem + (u == 0 ? TCU_N : 3 * TCU_N);
          const uint32_t acc = (ks == 0 && u <= 1) ? 0u : 1u;  // first write of each accumulator
          tc::mma_bf16(dre, are, bre, id_pos, acc);
          tc::mma_bf16(dre, aim, bim, id_neg, 1u);
          tc::mma_bf16(dim, are, bim, id_pos, acc);
          tc::mma_bf16(dim, aim, bre, id_pos, 1u);
        }
      }
    } else {
      s_ok = 0;
      tc::mbar_wait(&mbar_load, 0);  // let copies still in flight land before the CTA can exit
    }
    tc::commit(&mbar_mma);
  }
  // while the MMAs run: fetch this thread's row of the first 32 output columns
  const int i = i0 + warp * 32 + lane;
  cf cv[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    int j = j0 + c;
    cv[c] = (i < n && j < n) ? M[(size_t)j * n + i] : CF(0.f);
  }
  const bool done = tc::mbar_wait(&mbar_mma, 0);
  tc::fence_after();
  __syncthreads();
  const bool ok = done && s_ok;
  if (!ok && tid == 0 && err) atomicExch(err, 1);
  if (ok) {
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < TCU_N; c0 += 32) {
      if (c0 > 0) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          int j = j0 + c0 + c;
          cv[c] = (i < n && j < n) ? M[(size_t)j * n + i] : CF(0.f);
        }
      }
      float hr[32], hi[32], cr[32], ci[32];
      tc::tmem_ld32(tw + c0, hr);
      tc::tmem_ld32(tw + TCU_N + c0, hi);
      tc::tmem_ld32(tw + 2 * TCU_N + c0, cr);
      tc::tmem_ld32(tw + 3 * TCU_N + c0, ci);
      if (i < n) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          int j = j0 + c0 + c;
          if (j < n) M[(size_t)j * n + i] = CF(cv[c].x - (hr[c] + cr[c]), cv[c].y - (hi[c] + ci[c]));
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 4 * TCU_N);
}

template <class T>
static void lu_factor_impl(T* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm,
                           int* tc_err = nullptr, __nv_bfloat16* ws = nullptr) {
  cudaMemsetAsync(info, 0, sizeof(int) * batch, s);
  if constexpr (std::is_same<T, cf>::value)
    cudaFuncSetAttribute(gemm_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TCU_SMEM_LAUNCH);
  std::vector<cudaEvent_t> ev;
  int launches = 0;
  for (int k0 = 0; k0 < n; k0 += LU_NB) {
    int nbk = (n - k0 < LU_NB) ? n - k0 : LU_NB;
    if (!launch_panel_cluster<T>(A, n, k0, nbk, batch, piv, info, s))
      panel_kernel<T><<<batch, 1024, 0, s>>>(A, n, k0, nbk, piv, info);
    ++launches;
    int nother = n - nbk;
    if (nother > 0) { swap_kernel<T><<<dim3((nother + SWAP_COLS - 1) / SWAP_COLS, batch), 256, 0, s>>>(A, n, k0, nbk, piv); ++launches; }
    int rest = n - k0 - nbk;
    if (rest > 0) {
      trsm_kernel<T><<<dim3((rest + 127) / 128, batch), 128, 0, s>>>(A, n, k0, nbk);
      int t = (rest + GT - 1) / GT;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (tm) {
        cudaEventCreate(&e0); cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
      }
      if constexpr (std::is_same<T, cf>::value) {
        const int nL = (rest + TCU_M - 1) / TCU_M, nU = (rest + TCU_N - 1) / TCU_N;
        tcu_split_kernel<<<dim3(nL + nU, batch), 256, 0, s>>>((const cf*)A, n, k0, nbk, nL, ws);
        gemm_update_tc_kernel<<<dim3(nL, nU, batch), 128, TCU_SMEM_LAUNCH, s>>>((cf*)A, n, k0, nbk, ws, tc_err);
        ++launches;
      } else {
        gemm_update_kernel<T><<<dim3(t, t, batch), 256, 0, s>>>(A, n, k0, nbk);
      }
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

void lu_factor_batched_c64(cf* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm,
                           int* tc_err, void* ws) {
  lu_factor_impl<cf>(A, n, batch, piv, info, s, tm, tc_err, (__nv_bfloat16*)ws);
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
template <class TF, bool PHYS, int SGT>
__global__ void __launch_bounds__(256) solve_blocked_kernel(const TF* __restrict__ LU, const int* __restrict__ piv,
                                                            int n, int M, const double* __restrict__ sw,
                                                            const cd* __restrict__ rhs, cd* __restrict__ x,
                                                            int nrhs) {
  __shared__ TF Ls[SB][SB + 1];
  __shared__ TF Xs[SB][SGT];
  extern __shared__ int perm[];  // [n]: row interchanges composed into one permutation
  const int m = blockIdx.x;
  const int job0 = blockIdx.y * SGT;
  const int njobs_all = (m == 0) ? nrhs : 2 * nrhs;
  if (job0 >= njobs_all) return;
  const int G = min(SGT, njobs_all - job0);
  const TF* L = LU + (size_t)m * n * n;
  const int* pv = piv + (size_t)m * n;
  const int tid = threadIdx.x, T = blockDim.x;
  cd* X[SGT];
  for (int g = 0; g < SGT; ++g) {
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
      TF acc[SGT];
#pragma unroll
      for (int g = 0; g < SGT; ++g) acc[g] = czero<TF>();
      for (int c = 0; c < bs; ++c) {
        TF l = L[(size_t)(kb + c) * n + r];
#pragma unroll
        for (int g = 0; g < SGT; ++g) acc[g] = fma(l, Xs[c][g], acc[g]);
      }
#pragma unroll
      for (int g = 0; g < SGT; ++g)
        if (g < G) X[g][r] = X[g][r] - to_cd(acc[g]);
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
      TF acc[SGT];
#pragma unroll
      for (int g = 0; g < SGT; ++g) acc[g] = czero<TF>();
      for (int c = 0; c < bs; ++c) {
        TF u = L[(size_t)(kb + c) * n + r];
#pragma unroll
        for (int g = 0; g < SGT; ++g) acc[g] = fma(u, Xs[c][g], acc[g]);
      }
#pragma unroll
      for (int g = 0; g < SGT; ++g)
        if (g < G) X[g][r] = X[g][r] - to_cd(acc[g]);
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

// Vectors per CTA: 8, or 32 when that still leaves two CTAs per SM (many
// right-hand sides: every group reads the whole factor, so wider groups read
// it fewer times).
template <class TF, bool PHYS>
static void launch_solve_blocked(const TF* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x,
                                 int nrhs, cudaStream_t s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = n * (int)sizeof(int);
  const long long wide = (long long)(M + 1) * ((2 * nrhs + 31) / 32);
  if (wide >= 2LL * sms) {
    const int groups = (2 * nrhs + 31) / 32;
    cudaFuncSetAttribute(solve_blocked_kernel<TF, PHYS, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    solve_blocked_kernel<TF, PHYS, 32><<<dim3(M + 1, groups), 256, smem, s>>>(LU, piv, n, M, sw, rhs, x, nrhs);
  } else {
    const int groups = (2 * nrhs + SG - 1) / SG;
    cudaFuncSetAttribute(solve_blocked_kernel<TF, PHYS, SG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    solve_blocked_kernel<TF, PHYS, SG><<<dim3(M + 1, groups), 256, smem, s>>>(LU, piv, n, M, sw, rhs, x, nrhs);
  }
}

void lu_solve_modes(const cd* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x, int nrhs,
                    cudaStream_t s) {
  launch_solve_blocked<cd, true>(LU, piv, n, M, sw, rhs, x, nrhs, s);
}

void lu_correction_solve_c64(const cf* LU, const int* piv, int n, int M, const cd* r, cd* d, int nrhs,
                             cudaStream_t s) {
  launch_solve_blocked<cf, false>(LU, piv, n, M, nullptr, r, d, nrhs, s);
}
