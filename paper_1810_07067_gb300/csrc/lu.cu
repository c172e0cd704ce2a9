// Batched complex128 LU (right-looking, blocked by LU_NB columns) and solves.
//
// Per block column: (1) the panel is factored by one CTA per matrix with a
// warp-shuffle argmax for the pivot (largest |a|^2, lowest row on ties);
// (2) its row interchanges are applied to the other columns; (3) the block
// row of U is formed by a unit-lower triangular solve; (4) the trailing matrix
// is updated by a complex FP64 GEMM, batched over all matrices.
#include <algorithm>
#include <array>
#include <cstdio>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include "smem.cuh"
#include "lu.cuh"

std::mutex& lu_capture_mutex() {
  static std::mutex m;
  return m;
}
#include "tc.cuh"

namespace cg = cooperative_groups;

// Outer block of the complex64 factorization (see "two-level blocking" below).
#define LU_OB 128
#define LU_OB_CHUNKS (LU_OB / LU_NB)

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
__global__ void __launch_bounds__(1024) panel_kernel(const LuMat* __restrict__ mats, int k0) {
  const LuMat mat = mats[blockIdx.x];
  const int n = mat.n;
  if (k0 >= n) return;
  const int nbk = min(LU_NB, n - k0);
  T* M = (T*)mat.A;
  int* pv = mat.piv;
  int* info = mat.info;
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
        if (best <= V(0) && info[0] == 0) info[0] = c + 1;
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
// column-major slice [nbk][R].  Per column: local argmax; each CTA writes its
// candidate (value, row index and the row itself) into every CTA's shared
// memory through the cluster's distributed shared memory, and CTA 0, which
// owns row c whenever C > 1 (then R > LU_NB), writes row c as well; one
// cluster barrier; then every CTA picks the winner, the pivot's owner takes
// row c, CTA 0 takes the pivot row, and each CTA applies the rank-1 update to
// its rows.  Same pivot rule as panel_kernel (largest |a|^2, lowest row on
// ties).
#define PANEL_SMEM_MAX (200 * 1024)
#define PANEL_THREADS 512

template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) panel_cluster_kernel(const LuMat* __restrict__ mats, int k0, int R) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const LuMat mat = mats[blockIdx.y];  // the whole cluster works on one matrix
  const int n = mat.n;
  if (k0 >= n) return;                 // every CTA of the cluster, before any cluster barrier
  const int nbk = min(LU_NB, n - k0);
  T* M = (T*)mat.A;
  int* pv = mat.piv;
  int* info = mat.info;
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T* a = (T*)panel_smem;  // [nbk][R]
  using V = typename Pivot<T>::V;
  // exchange slots, double-buffered by column parity: a slot written for
  // column jj is written again only for column jj + 2, after every CTA has
  // passed the cluster barrier of column jj + 1 (so it has read it)
  __shared__ V cand_v[2][8];
  __shared__ int cand_i[2][8];
  __shared__ T cand_row[2][8][LU_NB];   // each CTA's candidate row of the panel
  __shared__ T top_row[2][LU_NB];       // row c (CTA 0 owns every row c of the panel)
  __shared__ V red_v[PANEL_THREADS / 32];
  __shared__ int red_i[PANEL_THREADS / 32];
  __shared__ int s_bi;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int row0 = k0 + q * R;
  const int nr = max(0, min(R, n - row0));  // rows owned by this CTA
  for (int t = tid; t < nbk * nr; t += PANEL_THREADS) {
    int r = t % nr, j = t / nr;
    a[j * R + r] = M[(size_t)(k0 + j) * n + row0 + r];
  }
  __syncthreads();
  for (int jj = 0; jj < nbk; ++jj) {
    const int c = k0 + jj, buf = jj & 1;
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
        cl.map_shared_rank(cand_v[buf], lane)[q] = best;
        cl.map_shared_rank(cand_i[buf], lane)[q] = bi;
      }
      if (lane == 0) s_bi = bi;
    }
    __syncthreads();
    // the candidate row (and, from CTA 0, row c) into every CTA
    const int cb = s_bi;
    if (tid < nbk * C) {
      const int j = tid % nbk, u = tid / nbk;
      if (cb < n) cl.map_shared_rank(cand_row[buf][q], u)[j] = a[j * R + cb - row0];
      if (q == 0) cl.map_shared_rank(top_row[buf], u)[j] = a[j * R + c - row0];
    }
    cl.sync();
    best = V(-1);
    bi = n;
    int win = -1;
    for (int u = 0; u < C; ++u) {
      const V v2 = cand_v[buf][u];
      const int i2 = cand_i[buf][u];
      if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; win = u; }
    }
    const int p = (best > V(0)) ? bi : -1;
    if (q == 0 && tid == 0) {
      pv[c] = (p >= 0) ? p : c;
      if (p < 0 && info[0] == 0) info[0] = c + 1;
    }
    if (p >= 0) {
      const T* prow = cand_row[buf][win];
      const int qp = (p - k0) / R;
      if (tid < nbk) {
        if (q == qp && p != c) a[tid * R + p - row0] = top_row[buf][tid];  // row c moves to p
        if (q == 0) a[tid * R + c - row0] = prow[tid];                       // the pivot row to c
      }
      __syncthreads();
      const T inv = cone<T>() / prow[jj];
      for (int r = max(0, c + 1 - row0) + tid; r < nr; r += PANEL_THREADS) {
        T l = a[jj * R + r] * inv;
        a[jj * R + r] = l;
        for (int j = jj + 1; j < nbk; ++j) a[j * R + r] = a[j * R + r] - l * prow[j];
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

// Cluster size: the smallest of 1, 2, 4, 8 whose row slices of the largest
// matrix (rows = its n - k0) fit PANEL_SMEM_MAX; smaller matrices of a ragged
// batch own fewer rows of the same slices.  Returns false (nothing launched)
// when none fits or no such cluster can be resident; the caller then uses
// panel_kernel.
template <class T>
static bool launch_panel_cluster(const LuMat* mats, int rows, int k0, int batch, cudaStream_t s) {
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
  if (cudaLaunchKernelEx(&cfg, panel_cluster_kernel<T>, mats, k0, R) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// ---------------------------------------------------------------- register panel
// Complex64 panel with the rows in registers: CTA q of a cluster of C owns
// rows k0 + q R .. k0 + (q+1) R - 1 (R = PREG_THREADS x PREG_RPT), thread t
// rows t + PREG_THREADS s (s < PREG_RPT), all LU_NB columns of each (the
// column loop is unrolled, so every register index is static).  Per column:
// local argmax (warp shuffles, then across the CTA's warps); the candidate
// row is staged in shared memory by its owner (and row c by its owner in CTA
// 0, which holds the panel's first R > LU_NB rows); every CTA's candidate
// (value, index, row) and row c reach every CTA through distributed shared
// memory (slots double-buffered by column parity); one cluster barrier; then
// each thread applies the interchange and the rank-1 update to its own rows.
// Same pivot rule and arithmetic as panel_cluster_kernel.
#define PREG_THREADS 256
#define PREG_RPT 2
#define PREG_R (PREG_THREADS * PREG_RPT)

struct PregShared {
  float cand_v[2][8];
  int cand_i[2][8];
  cf cand_row[2][8][LU_NB];  // each CTA's candidate row
  cf top_row[2][LU_NB];      // row c
  cf loc_row[LU_NB], loc_top[LU_NB];
  float red_v[PREG_THREADS / 32];
  int red_i[PREG_THREADS / 32];
};
struct PregCtx {
  int k0, n, nbk, C, q, tid, lane, wid;
  int* pv;
  int* info;
};

// Column jj of the panel.  The column loop is not unrolled (a fully unrolled
// panel overflows the instruction cache); every register access uses a
// compile-time column index, the column jj itself being picked out by a
// select over the 32 columns and the rank-1 update predicated on j > jj.
__device__ __forceinline__ void preg_column(int jj, const cg::cluster_group& cl, PregShared& sh, const PregCtx& x,
                                            cf (&a)[PREG_RPT][LU_NB], const int (&grow)[PREG_RPT]) {
  const int c = x.k0 + jj, buf = jj & 1, n = x.n;
  cf colv[PREG_RPT];
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s) {
    colv[s] = a[s][0];
#pragma unroll
    for (int j = 1; j < LU_NB; ++j)
      if (j == jj) colv[s] = a[s][j];
  }
  float best = -1.f;
  int bi = n;
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s)
    if (grow[s] >= c && grow[s] < n) argmax_merge(best, bi, Pivot<cf>::measure(colv[s]), grow[s]);
  for (int o = 16; o > 0; o >>= 1) {
    float v2 = __shfl_xor_sync(0xffffffffu, best, o);
    int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    argmax_merge(best, bi, v2, i2);
  }
  if (x.lane == 0) { sh.red_v[x.wid] = best; sh.red_i[x.wid] = bi; }
  __syncthreads();
  best = -1.f;
  bi = n;
#pragma unroll
  for (int w = 0; w < PREG_THREADS / 32; ++w) argmax_merge(best, bi, sh.red_v[w], sh.red_i[w]);
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s) {
    if (grow[s] == bi) {
#pragma unroll
      for (int j = 0; j < LU_NB; ++j) sh.loc_row[j] = a[s][j];
    }
    if (x.q == 0 && grow[s] == c) {
#pragma unroll
      for (int j = 0; j < LU_NB; ++j) sh.loc_top[j] = a[s][j];
    }
  }
  __syncthreads();
  if (x.tid < 32 * x.C) {
    const int j = x.tid & 31, u = x.tid >> 5;
    if (j < x.nbk) {
      if (bi < n) cl.map_shared_rank(&sh.cand_row[buf][x.q][0], u)[j] = sh.loc_row[j];
      if (x.q == 0) cl.map_shared_rank(&sh.top_row[buf][0], u)[j] = sh.loc_top[j];
    }
    if (j == 0) {
      cl.map_shared_rank(&sh.cand_v[buf][0], u)[x.q] = best;
      cl.map_shared_rank(&sh.cand_i[buf][0], u)[x.q] = bi;
    }
  }
  cl.sync();
  float bv = -1.f;
  int p = n, win = 0;
  for (int u = 0; u < x.C; ++u) {
    const float v2 = sh.cand_v[buf][u];
    const int i2 = sh.cand_i[buf][u];
    if (v2 > bv || (v2 == bv && i2 < p)) { bv = v2; p = i2; win = u; }
  }
  const bool ok = bv > 0.f;
  if (x.q == 0 && x.tid == 0) {
    x.pv[c] = ok ? p : c;
    if (!ok && x.info[0] == 0) x.info[0] = c + 1;
  }
  if (!ok) return;
  const cf* prow = sh.cand_row[buf][win];
  const cf* trow = sh.top_row[buf];
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s) {
    if (grow[s] == c) {  // row c takes the pivot row
#pragma unroll
      for (int j = 0; j < LU_NB; ++j) a[s][j] = prow[j];
    } else if (grow[s] == p) {  // the pivot's row takes row c
#pragma unroll
      for (int j = 0; j < LU_NB; ++j) a[s][j] = trow[j];
      colv[s] = trow[jj];
    }
  }
  const cf inv = cone<cf>() / prow[jj];
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s) {
    if (grow[s] > c && grow[s] < n) {
      const cf l = colv[s] * inv;
#pragma unroll
      for (int j = 0; j < LU_NB; ++j) {
        if (j > jj) a[s][j] = a[s][j] - l * prow[j];
        else if (j == jj) a[s][j] = l;
      }
    }
  }
}

__global__ void __launch_bounds__(PREG_THREADS, 1) panel_reg_kernel(const LuMat* __restrict__ mats, int k0) {
  cg::cluster_group cl = cg::this_cluster();
  const LuMat mat = mats[blockIdx.y];  // the whole cluster works on one matrix
  const int n = mat.n;
  if (k0 >= n) return;                 // every CTA of the cluster, before any cluster barrier
  __shared__ PregShared sh;
  PregCtx x;
  x.k0 = k0;
  x.n = n;
  x.nbk = min(LU_NB, n - k0);
  x.C = (int)cl.num_blocks();
  x.q = (int)cl.block_rank();
  x.tid = threadIdx.x;
  x.lane = threadIdx.x & 31;
  x.wid = threadIdx.x >> 5;
  x.pv = mat.piv;
  x.info = mat.info;
  cf* M = (cf*)mat.A;
  const int row0 = k0 + x.q * PREG_R;
  int grow[PREG_RPT];
  cf a[PREG_RPT][LU_NB];
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s) {
    grow[s] = row0 + x.tid + PREG_THREADS * s;
#pragma unroll
    for (int j = 0; j < LU_NB; ++j)
      a[s][j] = (grow[s] < n && j < x.nbk) ? M[(size_t)(k0 + j) * n + grow[s]] : CF(0.f);
  }
#pragma unroll 1
  for (int jj = 0; jj < x.nbk; ++jj) preg_column(jj, cl, sh, x, a, grow);
#pragma unroll
  for (int s = 0; s < PREG_RPT; ++s)
    if (grow[s] < n) {
#pragma unroll
      for (int j = 0; j < LU_NB; ++j)
        if (j < x.nbk) M[(size_t)(k0 + j) * n + grow[s]] = a[s][j];
    }
  cl.sync();  // no CTA leaves while a peer could still address its shared memory
}

// Cluster of C = ceil(rows / PREG_R) <= 8 CTAs; false when the panel is taller
// or no such cluster can be resident.
static bool launch_panel_reg(const LuMat* mats, int rows, int k0, int batch, cudaStream_t s) {
  const int C = (rows + PREG_R - 1) / PREG_R;
  if (C < 1 || C > 8) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, batch);
  cfg.blockDim = dim3(PREG_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, panel_reg_kernel, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  if (cudaLaunchKernelEx(&cfg, panel_reg_kernel, mats, k0) != cudaSuccess) {
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
//
// Columns (mode): 0 all but the panel's own; 1 those left of the panel and
// the rest of its LU_OB block (columns < min(K0 + LU_OB, n)); 2 those right
// of the block.
#define SWAP_COLS 64
template <class T>
__global__ void __launch_bounds__(256) swap_kernel(const LuMat* __restrict__ mats, int k0, int K0, int mode) {
  const LuMat mat = mats[blockIdx.y];
  const int n = mat.n;
  if (k0 >= n) return;
  const int nbk = min(LU_NB, n - k0);
  const int bend = min(K0 + LU_OB, n);
  const int lo = mode == 2 ? bend : 0, hi = mode == 1 ? bend : n;
  const bool skip = mode != 2;  // the panel's columns lie inside [lo, hi)
  const int ncols = hi - lo - (skip ? nbk : 0);
  const int* piv = mat.piv;
  __shared__ int pos[2 * LU_NB], src[2 * LU_NB], slot[LU_NB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kend = k0 + nbk;
  if (warp == 0) {
    const int p = (lane < nbk) ? piv[k0 + lane] : -1;
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
    const int idx = blockIdx.x * SWAP_COLS + cc;
    if (idx >= ncols) break;  // whole warp
    int c = lo + idx;
    if (skip && c >= k0) c += nbk;  // skip the panel's own columns
    T* col = (T*)mat.A + (size_t)c * n;
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
// Columns (mode): 0 all right of the panel; 1 those right of the panel
// inside its LU_OB block; 2 those right of the block.
template <class T>
__global__ void trsm_kernel(const LuMat* __restrict__ mats, int k0, int K0, int mode) {
  const LuMat mat = mats[blockIdx.y];
  const int n = mat.n;
  if (k0 + LU_NB >= n) return;  // no columns right of the panel (or the panel is the last)
  const int nbk = LU_NB;
  const int bend = min(K0 + LU_OB, n);
  const int clo = mode == 2 ? bend : k0 + nbk, chi = mode == 1 ? bend : n;
  T* M = (T*)mat.A;
  __shared__ T L[LU_NB][LU_NB + 1];
  for (int t = threadIdx.x; t < nbk * nbk; t += blockDim.x) {
    int r = t % nbk, cc = t / nbk;
    L[r][cc] = M[(size_t)(k0 + cc) * n + k0 + r];
  }
  __syncthreads();
  const int c = clo + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= chi) return;
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
__global__ void __launch_bounds__(256) gemm_update_kernel(const LuMat* __restrict__ mats, int k0) {
  const LuMat mat = mats[blockIdx.z];
  const int n = mat.n;
  const int nbk = LU_NB;
  const int start = k0 + nbk;
  if ((int)blockIdx.x * GT >= n - start || (int)blockIdx.y * GT >= n - start) return;
  T* M = (T*)mat.A;
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

// ---------------------------------------------------------------- two-level blocking (complex64)
// The complex64 factorization works on outer blocks of LU_OB = 4 LU_NB
// columns.  Inside a block, each LU_NB panel is factored, its interchanges
// are applied to the columns left of it and to the rest of the block, its
// rows of U are formed within the block, and the block's remaining columns
// are updated (all rows below: "R1").  Then the columns right of the block
// take the block's interchanges, in order, and the block's rows of U there
// are formed panel by panel (each panel's triangular solve followed by the
// update of the block's remaining rows: "R2").  Last, the trailing matrix
// right of and below the block ("R3") receives the four panels' updates
// together, as one rank-LU_OB product on the tensor cores, so it is read and
// written once per LU_OB columns instead of once per LU_NB.  (The columns
// right of the block must not take a panel's interchanges before the block
// is done: a row from below the block, without the deferred updates, would
// trade places with a row inside it, with them.)

// Strip update on the CUDA cores (FP32 arithmetic): C -= L U with
// L = A[r0..r1, k..k+LU_NB), U = A[k..k+LU_NB, c0..c1); which = 1 gives the
// block-column strip (rows k+LU_NB..n, columns k+LU_NB..min(K0+LU_OB, n)),
// which = 2 the block-row strip (rows k+LU_NB..min(K0+LU_OB, n), columns
// K0+LU_OB..n).  64 x 64 output tiles, 256 threads with 4 x 4 outputs each.
template <class T>
__global__ void __launch_bounds__(256) strip_update_kernel(const LuMat* __restrict__ mats, int K0, int k, int which) {
  const LuMat mat = mats[blockIdx.z];
  const int n = mat.n;
  if (k + LU_NB >= n) return;
  const int bend = min(K0 + LU_OB, n);
  const int r0 = k + LU_NB, r1 = which == 1 ? n : bend;
  const int c0 = which == 1 ? k + LU_NB : K0 + LU_OB, c1 = which == 1 ? bend : n;
  const int i0 = r0 + blockIdx.x * GT, j0 = c0 + blockIdx.y * GT;
  if (i0 >= r1 || j0 >= c1) return;
  T* M = (T*)mat.A;
  __shared__ T As[LU_NB][GT];
  __shared__ T Bs[LU_NB][GT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int t = tid; t < LU_NB * GT; t += 256) {
    const int r = t % GT, kk = t / GT;
    As[kk][r] = (i0 + r < r1) ? M[(size_t)(k + kk) * n + i0 + r] : czero<T>();
    const int kb = t % LU_NB, cj = t / LU_NB;
    Bs[kb][cj] = (j0 + cj < c1) ? M[(size_t)(j0 + cj) * n + k + kb] : czero<T>();
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = czero<T>();
#pragma unroll 4
  for (int kk = 0; kk < LU_NB; ++kk) {
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
    const int gj = j0 + ty + 16 * c;
    if (gj >= c1) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int gi = i0 + tx + 16 * a;
      if (gi < r1) {
        T* d = M + (size_t)gj * n + gi;
        *d = *d - acc[a][c];
      }
    }
  }
}

// Tensor-core update of R3: C -= L U with L = A[K0+LU_OB.., K0..K0+LU_OB) and
// U = A[K0..K0+LU_OB, K0+LU_OB..).  Every FP32 operand is split exactly into
// three BF16 pieces (x = hi + mid + lo, 24 bits), and the six piece products
// whose sum carries FP32 precision (hh, hm, mh, hl, mm, lh) are accumulated
// in FP32 tensor memory (-L_im U_im via the MMA's A-negation).  The hi*hi
// products and the five smaller corrections go to separate accumulators (Re
// and Im each, four in all) that are added in registers: sharing one
// accumulator loses about two bits to the tensor core's accumulation, which
// measured 4x the error of a plain FP32 update, while the split form measured
// half of it.  One CTA per 128 x TN output tile of one matrix; 128 threads;
// the operands arrive in LU_OB_CHUNKS chunks of LU_NB k-columns, each in the
// MMA's K-major no-swizzle core-matrix format, through one shared buffer.
#define TCU_M 128
#define TCU_ATILE (TCU_M * LU_NB)  // bf16 elements per piece chunk of an L tile (128 rows x 32 k)

// Column tile TN of the update: 32, 64 or 128 (chosen per block by the tile
// autotuner below).  The update kernel is persistent (one CTA per SM) and
// warp-specialised: a copy thread keeps a ring of NST operand chunks full, an
// MMA thread consumes them into one of NACC accumulator sets in tensor memory
// (4 TN columns each), and four epilogue warps apply a finished tile to C
// while the MMAs of the next tile run.
template <int TN> struct TcuShape {
  static constexpr int BTILE = TN * LU_NB;                        // bf16 elements per piece chunk of a U tile
  static constexpr int STAGE = 6 * (TCU_ATILE + BTILE) * 2;       // one chunk of both operands, six pieces each
  static constexpr int NST = (3 * STAGE <= 220 * 1024) ? 3 : 2;
  static constexpr int SMEM = NST * STAGE;
  static constexpr uint32_t SET_COLS = 4 * TN;
  static constexpr int NACC = (2 * SET_COLS <= 512) ? 2 : 1;
  static constexpr uint32_t TMEM_COLS = NACC * SET_COLS <= 256 ? 256 : 512;
};

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

// Workspace of one matrix: the L block column (rows K0+LU_OB.., LU_OB
// k-columns) and the U block row (LU_OB k-rows, columns K0+LU_OB..) split
// into their BF16 pieces, stored tile by tile in exactly the shared-memory
// image the MMAs read: ceil(n/128) L tiles of [LU_OB_CHUNKS][6 pieces][128 x 32],
// then ceil(n/TN) U tiles of [LU_OB_CHUNKS][6][TN x 32] (room for ceil(n/128)
// tiles of 128 columns, the largest TN).
__host__ __device__ inline size_t tcu_ws_matrix_elems(int n) {
  return (size_t)((n + TCU_M - 1) / TCU_M) * LU_OB_CHUNKS * 6 * (TCU_ATILE + 128 * LU_NB);
}

size_t lu_c64_workspace_bytes(int n, int batch) { return tcu_ws_matrix_elems(n) * (size_t)batch * 2; }

template <int TN>
__global__ void __launch_bounds__(256) tcu_split_kernel(const LuMat* __restrict__ mats, int K0, int nL) {
  using S = TcuShape<TN>;
  const LuMat mat = mats[blockIdx.y];
  const int n = mat.n;
  const int start = K0 + LU_OB, rest = n - start;
  if (rest <= 0) return;
  const cf* M = (const cf*)mat.A;
  __nv_bfloat16* W = (__nv_bfloat16*)mat.ws;
  // thread item: one row (of L) or column (of U) and 8 consecutive k, written
  // as one 16-byte core-matrix row per piece
  auto put = [&](__nv_bfloat16* d, int stride, const cf* v) {
    __align__(16) __nv_bfloat16 pc[6][8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      __nv_bfloat16 pr[3], pi[3];
      split3(v[c].x, pr); split3(v[c].y, pi);
#pragma unroll
      for (int q = 0; q < 3; ++q) { pc[q][c] = pr[q]; pc[3 + q][c] = pi[q]; }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) *(uint4*)(d + (size_t)q * stride) = *(const uint4*)pc[q];
  };
  if ((int)blockIdx.x < nL) {
    if ((int)blockIdx.x * TCU_M >= rest) return;
    const int r0 = start + blockIdx.x * TCU_M;
    __nv_bfloat16* dst = W + (size_t)blockIdx.x * LU_OB_CHUNKS * 6 * TCU_ATILE;
    for (int t = threadIdx.x; t < TCU_M * (LU_OB / 8); t += 256) {
      const int r = t % TCU_M, kb0 = (t / TCU_M) * 8, ch = kb0 / LU_NB, k0 = kb0 % LU_NB;
      cf v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = (r0 + r < n) ? M[(size_t)(K0 + kb0 + c) * n + r0 + r] : CF(0.f);
      put(dst + (size_t)ch * 6 * TCU_ATILE + tcu_off(r, k0), TCU_ATILE, v);
    }
  } else {
    const int y = blockIdx.x - nL;
    if (y * TN >= rest) return;
    const int c0 = start + y * TN;
    __nv_bfloat16* dst = W + (size_t)((n + TCU_M - 1) / TCU_M) * LU_OB_CHUNKS * 6 * TCU_ATILE +
                         (size_t)y * LU_OB_CHUNKS * 6 * S::BTILE;
    for (int t = threadIdx.x; t < TN * (LU_OB / 8); t += 256) {
      const int kb0 = (t % (LU_OB / 8)) * 8, j = t / (LU_OB / 8), ch = kb0 / LU_NB, k0 = kb0 % LU_NB;
      cf v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = (c0 + j < n) ? M[(size_t)(c0 + j) * n + K0 + kb0 + c] : CF(0.f);
      put(dst + (size_t)ch * 6 * S::BTILE + tcu_off(j, k0), S::BTILE, v);
    }
  }
}

// Persistent update over the tiles of every matrix of the launch: tile t =
// (matrix z, column tile y, row tile x), x fastest, taken by CTA t mod
// gridDim.x; tiles outside a matrix's own trailing block are skipped by all
// three roles alike.  Every wait is bounded: a role that gives up sets the
// CTA's failure flag (and *err), the others stop at their next wait, and
// before the CTA exits the copy thread lets its copies in flight land and the
// MMA thread waits for its MMAs.
template <int TN>
__global__ void __launch_bounds__(192, 1) gemm_update_tc_kernel(const LuMat* __restrict__ mats, int K0, int nLmax,
                                                               int nUmax, int count, int* __restrict__ err) {
  using S = TcuShape<TN>;
  constexpr int NST = S::NST, NACC = S::NACC;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[NST], empty[NST], tfull[NACC], tempty[NACC], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  volatile int* fail = &s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int start = K0 + LU_OB;
  const long long per = (long long)nLmax * nUmax, total = per * count;
  auto tile_of = [&](long long t, int& z, int& x, int& y) -> bool {
    z = (int)(t / per);
    const long long r = t - (long long)z * per;
    y = (int)(r / nLmax);
    x = (int)(r - (long long)y * nLmax);
    const int rest = mats[z].n - start;
    return x * TCU_M < rest && y * TN < rest;
  };
  if (warp == 0) tc::tmem_alloc(&tmem_base, S::TMEM_COLS);
  if (tid == 32) {
    s_fail = 0;
#pragma unroll
    for (int b = 0; b < NST; ++b) { tc::mbar_init(&full[b], 1); tc::mbar_init(&empty[b], 1); }
#pragma unroll
    for (int b = 0; b < NACC; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 4); }
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;  // copy thread: chunks whose copies were issued
  if (warp == 4) {
    if (lane == 0) {
      int q = 0;
      for (long long t = blockIdx.x; t < total && !*fail; t += gridDim.x) {
        int z, x, y;
        if (!tile_of(t, z, x, y)) continue;
        const int n = mats[z].n;
        const __nv_bfloat16* W = (const __nv_bfloat16*)mats[z].ws;
        const __nv_bfloat16* Lsrc = W + (size_t)x * LU_OB_CHUNKS * 6 * TCU_ATILE;
        const __nv_bfloat16* Usrc = W + (size_t)((n + TCU_M - 1) / TCU_M) * LU_OB_CHUNKS * 6 * TCU_ATILE +
                                    (size_t)y * LU_OB_CHUNKS * 6 * S::BTILE;
        for (int ch = 0; ch < LU_OB_CHUNKS; ++ch, ++q) {
          const int st = q % NST;
          if (q >= NST && !tc::mbar_wait(&empty[st], ((q / NST) - 1) & 1)) { *fail = 1; break; }
          unsigned char* base = smem + (size_t)st * S::STAGE;
          tc::mbar_expect_tx(&full[st], S::STAGE);
          tc::bulk_g2s(base, Lsrc + (size_t)ch * 6 * TCU_ATILE, 6 * TCU_ATILE * 2, &full[st]);
          tc::bulk_g2s(base + 6 * TCU_ATILE * 2, Usrc + (size_t)ch * 6 * S::BTILE, 6 * S::BTILE * 2, &full[st]);
          issued = q + 1;
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t id_pos = tc::idesc_bf16_f32(TCU_M, TN, false);
      const uint32_t id_neg = tc::idesc_bf16_f32(TCU_M, TN, true);
      const uint64_t at = (uint64_t)(TCU_ATILE * 2 / 16), bt = (uint64_t)(S::BTILE * 2 / 16);  // 16-byte units
      const int qa_[6] = {0, 0, 1, 0, 1, 2}, qb_[6] = {0, 1, 0, 2, 1, 0};
      int q = 0, k = 0;
      for (long long t = blockIdx.x; t < total && !*fail; t += gridDim.x) {
        int z, x, y;
        if (!tile_of(t, z, x, y)) continue;
        const int set = k % NACC;
        if (k >= NACC && !tc::mbar_wait(&tempty[set], ((k / NACC) - 1) & 1)) { *fail = 1; break; }
        tc::fence_after();
        // accumulator columns of the set: [0,TN) hh Re, [TN,2TN) hh Im, [2TN,3TN) corrections Re, [3TN,4TN) Im
        const uint32_t d0 = tmem + (uint32_t)set * S::SET_COLS;
        for (int ch = 0; ch < LU_OB_CHUNKS; ++ch, ++q) {
          const int st = q % NST;
          if (!tc::mbar_wait(&full[st], (q / NST) & 1)) { *fail = 1; break; }
          tc::fence_after();
          unsigned char* base = smem + (size_t)st * S::STAGE;
          const uint64_t a0 = tc::desc_noswizzle(tc::smem_u32(base), 128, (LU_NB / 8) * 128);
          const uint64_t b0 = tc::desc_noswizzle(tc::smem_u32(base + 6 * TCU_ATILE * 2), 128, (LU_NB / 8) * 128);
#pragma unroll
          for (int ks = 0; ks < LU_NB / 16; ++ks) {
            const uint64_t kof = (uint64_t)(ks * 256 / 16);  // two core matrices along k
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              const uint64_t are = a0 + qa_[u] * at + kof, aim = a0 + (3 + qa_[u]) * at + kof;
              const uint64_t bre = b0 + qb_[u] * bt + kof, bim = b0 + (3 + qb_[u]) * bt + kof;
              const uint32_t dre = d0 + (u == 0 ? 0 : 2 * TN), dim = d0 + (u == 0 ? TN : 3 * TN);
              const uint32_t acc = (ch == 0 && ks == 0 && u <= 1) ? 0u : 1u;  // first write of each accumulator
              tc::mma_bf16(dre, are, bre, id_pos, acc);
              tc::mma_bf16(dre, aim, bim, id_neg, 1u);
              tc::mma_bf16(dim, are, bim, id_pos, acc);
              tc::mma_bf16(dim, aim, bre, id_pos, 1u);
            }
          }
          tc::commit(&empty[st]);  // the stage is free once these MMAs have read it
        }
        if (*fail) break;
        tc::commit(&tfull[set]);   // the tile's accumulators are complete
        ++k;
      }
      tc::commit(&mdone);          // arrives once every MMA issued above has completed
      if (!tc::mbar_wait(&mdone, 0)) *fail = 1;
    }
  } else {
    // epilogue warps: warp w owns tensor-memory lanes (tile rows) 32w .. 32w + 31
    int k = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
      int z, x, y;
      if (!tile_of(t, z, x, y)) continue;
      const int set = k % NACC;
      const int n = mats[z].n;
      cf* M = (cf*)mats[z].A;
      const int i = start + x * TCU_M + warp * 32 + lane, j0 = start + y * TN;
      cf cv[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {  // C of the first 32 columns while the MMAs run
        const int j = j0 + c;
        cv[c] = (i < n && j < n) ? M[(size_t)j * n + i] : CF(0.f);
      }
      if (!tc::mbar_wait(&tfull[set], (k / NACC) & 1)) { *fail = 1; break; }
      tc::fence_after();
      const uint32_t tw = tmem + (uint32_t)set * S::SET_COLS + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 32) {
        if (c0 > 0) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int j = j0 + c0 + c;
            cv[c] = (i < n && j < n) ? M[(size_t)j * n + i] : CF(0.f);
          }
        }
        float h[32], e[32];  // Re parts into cv first, then Im: two accumulator pairs live at a time
        tc::tmem_ld32(tw + c0, h);
        tc::tmem_ld32(tw + 2 * TN + c0, e);
#pragma unroll
        for (int c = 0; c < 32; ++c) cv[c].x -= h[c] + e[c];
        tc::tmem_ld32(tw + TN + c0, h);
        tc::tmem_ld32(tw + 3 * TN + c0, e);
#pragma unroll
        for (int c = 0; c < 32; ++c) cv[c].y -= h[c] + e[c];
        if (i < n) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int j = j0 + c0 + c;
            if (j < n) M[(size_t)j * n + i] = cv[c];
          }
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[set]);
      ++k;
    }
  }
  __syncthreads();
  if (*fail) {
    if (tid == 0 && err) atomicExch(err, 1);
    if (warp == 4 && lane == 0) {
      // let the copies still in flight land before the CTA exits (bounded):
      // the newest copy of each stage completes the newest phase of its barrier
      for (int st = 0; st < NST; ++st) {
        const int last = issued - 1 - ((issued - 1 - st) % NST + NST) % NST;  // newest chunk issued into st
        if (last >= 0) tc::mbar_wait(&full[st], (last / NST) & 1, 1 << 20);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

// ---------------------------------------------------------------- driver
static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 1;
  }
  return sms;
}

// R3 of outer block K0 for the matrices 0..active-1 (those with n > K0 + LU_OB);
// rest = nmax - K0 - LU_OB is the largest trailing size.
template <int TN>
static void tc_update_tn(const LuMat* d, int K0, int rest, int active, int* tc_err, cudaStream_t s) {
  const int nL = (rest + TCU_M - 1) / TCU_M, nU = (rest + TN - 1) / TN;
  tcu_split_kernel<TN><<<dim3(nL + nU, active), 256, 0, s>>>(d, K0, nL);
  const long long tiles = (long long)nL * nU * active;
  const int grid = (int)std::min<long long>(tiles, sm_count());
  gemm_update_tc_kernel<TN><<<grid, 192, TcuShape<TN>::SMEM, s>>>(d, K0, nL, nU, active, tc_err);
}

static void tc_update(int tn, const LuMat* d, int K0, int rest, int active, int* tc_err, cudaStream_t s) {
  if (tn == 32) tc_update_tn<32>(d, K0, rest, active, tc_err, s);
  else if (tn == 128) tc_update_tn<128>(d, K0, rest, active, tc_err, s);
  else tc_update_tn<64>(d, K0, rest, active, tc_err, s);
}

static void tc_set_attributes() {
  cudaFuncSetAttribute(gemm_update_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcuShape<32>::SMEM);
  cudaFuncSetAttribute(gemm_update_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcuShape<64>::SMEM);
  cudaFuncSetAttribute(gemm_update_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcuShape<128>::SMEM);
}

__global__ void lu_info_zero_kernel(const LuMat* __restrict__ mats, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < count) mats[b].info[0] = 0;
}

// Tile autotuner.  The column tile TN of the tensor-core update is chosen per
// LU step from the trailing size (rest) and the number of matrices in the
// launch.  For each power-of-two bucket of rest ((64, 128], (128, 256], ...,
// above 8192) and of the matrix count, the split + update pair is timed once
// per process on scratch matrices of the bucket's middle size with TN = 32, 64
// and 128 (CUDA events on the caller's stream, best of three after one
// warm-up); the tile with the least time per matrix is kept, TN = 64 unless
// another is at least 3 % faster.  Scratch is capped near 1 GiB by timing
// fewer matrices of large sizes (their launches still fill the GPU).
namespace {
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tune;
std::map<std::pair<int, int>, std::array<float, 3>> g_tune_ms;
int rest_bucket(int rest) { int b = 0; while (b < 7 && (128 << b) < rest) ++b; return b; }
int count_bucket(int c) { int b = 0; while (b < 16 && (1 << b) < c) ++b; return b; }
}  // namespace

__global__ void tune_fill_kernel(cf* A, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)(i >> 32);
    h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
    A[i] = CF((float)(h & 0xffff) * (2.f / 65535.f) - 1.f, (float)(h >> 16) * (2.f / 65535.f) - 1.f);
  }
}

static int measure_tile(int R, int count, cudaStream_t s, std::array<float, 3>& ms) {
  const int n = R + LU_OB;
  const size_t elems = (size_t)n * n, wse = tcu_ws_matrix_elems(n);
  const size_t per = elems * sizeof(cf) + wse * 2;
  const int c = (int)std::min<size_t>((size_t)count, std::max<size_t>(1, ((size_t)1 << 30) / per));
  cf* A = nullptr;
  __nv_bfloat16* ws = nullptr;
  LuMat* d = nullptr;
  int* err = nullptr;
  ms = {-1.f, -1.f, -1.f};
  if (cudaMallocAsync((void**)&A, elems * c * sizeof(cf), s) != cudaSuccess ||
      cudaMallocAsync((void**)&ws, wse * c * 2, s) != cudaSuccess ||
      cudaMallocAsync((void**)&d, sizeof(LuMat) * c, s) != cudaSuccess ||
      cudaMallocAsync((void**)&err, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    if (A) cudaFreeAsync(A, s);
    if (ws) cudaFreeAsync(ws, s);
    if (d) cudaFreeAsync(d, s);
    if (err) cudaFreeAsync(err, s);
    return 64;
  }
  std::vector<LuMat> it(c);
  for (int i = 0; i < c; ++i) it[i] = LuMat{A + elems * i, nullptr, nullptr, ws + wse * i, n, 0};
  cudaMemcpyAsync(d, it.data(), sizeof(LuMat) * c, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(err, 0, sizeof(int), s);
  tune_fill_kernel<<<1024, 256, 0, s>>>(A, elems * c);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  const int tns[3] = {32, 64, 128};
  for (int q = 0; q < 3; ++q) {
    tc_update(tns[q], d, 0, R, c, err, s);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      tc_update(tns[q], d, 0, R, c, err, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, t);
    }
    ms[q] = best / c;
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  cudaFreeAsync(A, s); cudaFreeAsync(ws, s); cudaFreeAsync(d, s); cudaFreeAsync(err, s);
  if (cudaGetLastError() != cudaSuccess || herr) return 64;
  int pick = 1;
  for (int q : {0, 2})
    if (ms[q] > 0.f && ms[q] < 0.97f * ms[pick]) pick = q;
  return tns[pick];
}

static void autotune_tiles(int nmax, int count, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int cb = count_bucket(count);
  for (int rb = 0; rb <= rest_bucket(nmax - LU_OB); ++rb) {
    if (g_tune.count({rb, cb})) continue;
    std::array<float, 3> ms;
    const int tn = measure_tile(96 << rb, count, s, ms);  // the bucket's middle trailing size
    g_tune[{rb, cb}] = tn;
    g_tune_ms[{rb, cb}] = ms;
  }
}

static int tuned_tile(int rest, int count) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto f = g_tune.find({rest_bucket(rest), count_bucket(count)});
  return f == g_tune.end() ? 64 : f->second;
}

int lu_tile_table(int* rest_hi, int* count_hi, int* tile, float* ms, int cap) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int k = 0;
  for (const auto& e : g_tune) {
    if (k >= cap) break;
    rest_hi[k] = 128 << e.first.first;
    count_hi[k] = 1 << e.first.second;
    tile[k] = e.second;
    const auto& m = g_tune_ms[e.first];
    for (int q = 0; q < 3; ++q) ms[3 * k + q] = m[q];
    ++k;
  }
  return k;
}

// Right-looking blocked LU of every matrix of the table, largest first: at
// step k0 the launches cover the matrices with n > k0 (a prefix of the sorted
// table), each kernel reading its matrix, size and pivots from the table.
template <class T>
static cudaError_t lu_factor_impl(const LuMat* items, int count, cudaStream_t s, LuTiming* tm, int* tc_err, int tile,
                                  bool graph) {
  if (count <= 0) return cudaSuccess;
  std::vector<LuMat> it(items, items + count);
  std::stable_sort(it.begin(), it.end(), [](const LuMat& a, const LuMat& b) { return a.n > b.n; });
  const int nmax = it[0].n;
  LuMat* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, sizeof(LuMat) * count, s);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(d, it.data(), sizeof(LuMat) * count, cudaMemcpyHostToDevice, s);
  lu_info_zero_kernel<<<(count + 255) / 256, 256, 0, s>>>(d, count);
  constexpr bool c64 = std::is_same<T, cf>::value;
  if constexpr (c64) {
    tc_set_attributes();
    if (tile == 0) autotune_tiles(nmax, count, s);
  }
  cudaStream_t ls = s, cs = nullptr;
  // while this thread captures, no other thread of the library frees device
  // memory (a free synchronizes the device, which would end the capture)
  std::unique_lock<std::mutex> capture_lock(lu_capture_mutex(), std::defer_lock);
  if (graph) capture_lock.lock();
  if (graph) {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      if (cs) cudaStreamDestroy(cs);
      cs = nullptr;
      graph = false;
      capture_lock.unlock();
    } else {
      ls = cs;
    }
  }
  const bool timed = tm && !graph;
  std::vector<cudaEvent_t> ev;
  int launches = 1, gemm_launches = 0, tn_steps[3] = {0, 0, 0};
  double gemm_flops = 0.0, gemm_bytes = 0.0;
  int active = count;
  auto timed_launch = [&](auto&& launch) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
      cudaEventCreate(&e0); cudaEventCreate(&e1);
      cudaEventRecord(e0, ls);
    }
    launch();
    if (timed) {
      cudaEventRecord(e1, ls);
      ev.push_back(e0); ev.push_back(e1);
    }
  };
  // one LU_NB panel at column k0: factor, interchange, rows of U right of it
  // (mode 0: all columns; mode 1: within the LU_OB block starting at K0)
  auto panel_step = [&](int k0, int K0, int mode) -> int {
    while (active > 0 && it[active - 1].n <= k0) --active;
    const int nbk = std::min(LU_NB, nmax - k0);
    bool done = false;
    if constexpr (c64) done = launch_panel_reg(d, nmax - k0, k0, active, ls);
    if (!done && !launch_panel_cluster<T>(d, nmax - k0, k0, active, ls)) panel_kernel<T><<<active, 1024, 0, ls>>>(d, k0);
    ++launches;
    const int hi = mode == 1 ? std::min(K0 + LU_OB, nmax) : nmax;
    if (hi - nbk > 0) {
      swap_kernel<T><<<dim3((hi - nbk + SWAP_COLS - 1) / SWAP_COLS, active), 256, 0, ls>>>(d, k0, K0, mode);
      ++launches;
    }
    const int rest = hi - k0 - nbk;
    if (rest > 0) {
      trsm_kernel<T><<<dim3((rest + 127) / 128, active), 128, 0, ls>>>(d, k0, K0, mode);
      ++launches;
    }
    return rest;
  };
  if constexpr (c64) {
    // two-level: LU_NB panels inside LU_OB blocks, one rank-LU_OB tensor-core update per block
    for (int K0 = 0; K0 < nmax; K0 += LU_OB) {
      for (int p = 0; p < LU_OB_CHUNKS; ++p) {
        const int k0 = K0 + p * LU_NB;
        if (k0 >= nmax) break;
        const int bcols = panel_step(k0, K0, 1);                    // R1: block columns right of the panel
        if (bcols <= 0) continue;
        const int rows = nmax - k0 - LU_NB;
        strip_update_kernel<T><<<dim3((rows + GT - 1) / GT, (bcols + GT - 1) / GT, active), 256, 0, ls>>>(
            d, K0, k0, 1);
        ++launches;
      }
      const int rest = nmax - K0 - LU_OB;                           // columns right of the block
      if (rest <= 0) continue;
      int a3 = active;                                               // the matrices that have them
      while (a3 > 0 && it[a3 - 1].n <= K0 + LU_OB) --a3;
      if (a3 <= 0) continue;
      for (int p = 0; p < LU_OB_CHUNKS; ++p) {                      // the block's interchanges, in order
        swap_kernel<T><<<dim3((rest + SWAP_COLS - 1) / SWAP_COLS, a3), 256, 0, ls>>>(d, K0 + p * LU_NB, K0, 2);
        ++launches;
      }
      for (int p = 0; p < LU_OB_CHUNKS; ++p) {                      // rows of U right of the block; R2
        const int k0 = K0 + p * LU_NB;
        trsm_kernel<T><<<dim3((rest + 127) / 128, a3), 128, 0, ls>>>(d, k0, K0, 2);
        ++launches;
        const int brows = LU_OB - (p + 1) * LU_NB;
        if (brows > 0) {
          strip_update_kernel<T><<<dim3((brows + GT - 1) / GT, (rest + GT - 1) / GT, a3), 256, 0, ls>>>(
              d, K0, k0, 2);
          ++launches;
        }
      }
      // R3
      const int tn = tile ? tile : tuned_tile(rest, a3);
      timed_launch([&] { tc_update(tn, d, K0, rest, a3, tc_err, ls); });
      ++tn_steps[tn == 32 ? 0 : tn == 64 ? 1 : 2];
      launches += 2;
      for (int b = 0; b < a3; ++b) {
        const double rb = (double)(it[b].n - K0 - LU_OB);
        if (rb > 0) {
          gemm_flops += 8.0 * rb * rb * LU_OB;
          gemm_bytes += 2.0 * sizeof(T) * rb * rb;   // the trailing matrix read and written once
        }
      }
      ++gemm_launches;
    }
  } else {
    for (int k0 = 0; k0 < nmax; k0 += LU_NB) {
      const int rest = panel_step(k0, 0, 0);
      if (rest <= 0) continue;
      const int t = (rest + GT - 1) / GT;
      timed_launch([&] { gemm_update_kernel<T><<<dim3(t, t, active), 256, 0, ls>>>(d, k0); });
      ++launches;
      for (int b = 0; b < active; ++b) {
        const double rb = (double)(it[b].n - k0 - LU_NB);
        if (rb > 0) {
          gemm_flops += 8.0 * rb * rb * LU_NB;
          gemm_bytes += 2.0 * sizeof(T) * rb * rb;
        }
      }
      ++gemm_launches;
    }
  }
  if (graph) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    capture_lock.unlock();
    if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, s);
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {  // nothing of the capture ran: factor with direct launches instead
      cudaGetLastError();
      cudaFreeAsync(d, s);
      return lu_factor_impl<T>(items, count, s, tm, tc_err, tile, false);
    }
  }
  cudaFreeAsync(d, s);
  if (tm) {
    tm->launches += launches;
    tm->gemm_flops += gemm_flops;
    tm->gemm_bytes += gemm_bytes;
    tm->gemm_launches += gemm_launches;
    tm->graph = graph ? 1 : 0;
    for (int q = 0; q < 3; ++q) tm->tile_steps[q] += tn_steps[q];
    if (!ev.empty()) cudaEventSynchronize(ev.back());
    for (size_t q = 0; q + 1 < ev.size(); q += 2) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
      tm->gemm_ms += ms;
      cudaEventDestroy(ev[q]); cudaEventDestroy(ev[q + 1]);
    }
  }
  return cudaGetLastError();
}

cudaError_t lu_factor_many(const LuMat* items, int count, bool c64, cudaStream_t s, LuTiming* tm, int* tc_err,
                           int tile, bool graph) {
  return c64 ? lu_factor_impl<cf>(items, count, s, tm, tc_err, tile, graph)
             : lu_factor_impl<cd>(items, count, s, tm, nullptr, 0, graph);
}

void lu_factor_batched(cd* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm) {
  std::vector<LuMat> it(batch);
  for (int b = 0; b < batch; ++b) it[b] = LuMat{A + (size_t)b * n * n, piv + (size_t)b * n, info + b, nullptr, n, 0};
  lu_factor_impl<cd>(it.data(), batch, s, tm, nullptr, 0, false);
}

void lu_factor_batched_c64(cf* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* tm,
                           int* tc_err, void* ws, int tile) {
  std::vector<LuMat> it(batch);
  for (int b = 0; b < batch; ++b)
    it[b] = LuMat{A + (size_t)b * n * n, piv + (size_t)b * n, info + b,
                  (__nv_bfloat16*)ws + tcu_ws_matrix_elems(n) * b, n, 0};
  lu_factor_impl<cf>(it.data(), batch, s, tm, tc_err, tile, false);
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
//
// Schedule of one pass (forward shown; the backward pass mirrors it): with
// block i solved (its x in Xs[i & 1]), threads 0..63 update the rows of block
// i+1 with block i's factor column, then warp 0 solves block i+1's diagonal
// triangle in registers (rows lane and lane + 32, broadcast by shuffles),
// while the other threads load the diagonal block i+2 into shared memory and
// update every row beyond block i+1 (a streaming product, eight factor
// columns in flight per thread): the triangle is off the critical path.
template <int SGT> struct SolveShape { static constexpr int NT = SGT <= 4 ? 512 : 256; };

template <class T> __device__ __forceinline__ T shfl_c(T v, int src) {
  T r;
  r.x = __shfl_sync(0xffffffffu, v.x, src);
  r.y = __shfl_sync(0xffffffffu, v.y, src);
  return r;
}

// Warp 0: the diagonal triangle of the block at rows kb.. (bs rows) for all
// G jobs, JC at a time (2 under the 64-register cap of 1024-thread CTAs);
// unit lower (FWD) or upper with its diagonal.  The solution goes to Xo
// (shared, for the block's column product) and to X.
template <class TF, int SGT, bool FWD, int JC = (SolveShape<SGT>::NT >= 1024 ? 2 : 4)>
__device__ __forceinline__ void warp_triangle(const TF (*Lb)[SB + 1], TF (*Xo)[SGT], cd* const* X, int kb, int bs,
                                              int G, int lane) {
  for (int g0 = 0; g0 < G; g0 += JC) {
    TF xv[2][JC];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = lane + 32 * s;
#pragma unroll
      for (int gg = 0; gg < JC; ++gg)
        xv[s][gg] = (r < bs && g0 + gg < G) ? conv<TF>(X[g0 + gg][kb + r]) : czero<TF>();
    }
    if (FWD) {
      for (int c = 0; c < bs - 1; ++c) {
        const int owner = c & 31;
        TF xc[JC];
#pragma unroll
        for (int gg = 0; gg < JC; ++gg) xc[gg] = shfl_c(c < 32 ? xv[0][gg] : xv[1][gg], owner);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int r = lane + 32 * s;
          if (r > c && r < bs) {
            const TF l = Lb[r][c];
#pragma unroll
            for (int gg = 0; gg < JC; ++gg) xv[s][gg] = xv[s][gg] - l * xc[gg];
          }
        }
      }
    } else {
      for (int c = bs - 1; c >= 0; --c) {
        const int owner = c & 31, slot = c >> 5;
        const TF d = Lb[c][c];
        TF xc[JC];
#pragma unroll
        for (int gg = 0; gg < JC; ++gg) xc[gg] = shfl_c(slot ? xv[1][gg] : xv[0][gg], owner) / d;
        if (lane == owner) {
#pragma unroll
          for (int gg = 0; gg < JC; ++gg) {
            if (slot) xv[1][gg] = xc[gg];
            else xv[0][gg] = xc[gg];
          }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int r = lane + 32 * s;
          if (r < c) {
            const TF u = Lb[r][c];
#pragma unroll
            for (int gg = 0; gg < JC; ++gg) xv[s][gg] = xv[s][gg] - u * xc[gg];
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = lane + 32 * s;
#pragma unroll
      for (int gg = 0; gg < JC; ++gg)
        if (r < bs && g0 + gg < G) {
          Xo[r][g0 + gg] = xv[s][gg];
          X[g0 + gg][kb + r] = to_cd(xv[s][gg]);
        }
    }
  }
}

// x_r -= sum_c F[r, kb + c] x_c over the bs columns of one block (x_c in Xb).
template <class TF, int SGT>
__device__ __forceinline__ void block_row_update(const TF* __restrict__ F, int n, int r, int kb, int bs,
                                                 const TF (*Xb)[SGT], cd* const* X, int G) {
  TF acc[SGT];
#pragma unroll
  for (int g = 0; g < SGT; ++g) acc[g] = czero<TF>();
#pragma unroll 8
  for (int c = 0; c < bs; ++c) {
    const TF l = F[(size_t)(kb + c) * n + r];
#pragma unroll
    for (int g = 0; g < SGT; ++g) acc[g] = fma(l, Xb[c][g], acc[g]);
  }
#pragma unroll
  for (int g = 0; g < SGT; ++g)
    if (g < G) X[g][r] = X[g][r] - to_cd(acc[g]);
}

// The same for rows r and r + 1 (r even, both below the matrix's end): one
// 16-byte load per factor column feeds both rows (more bytes in flight per
// thread on this bandwidth-bound product).
template <int SGT>
__device__ __forceinline__ void block_row_update2(const cf* __restrict__ F, int n, int r, int kb, int bs,
                                                  const cf (*Xb)[SGT], cd* const* X, int G) {
  cf acc0[SGT], acc1[SGT];
#pragma unroll
  for (int g = 0; g < SGT; ++g) { acc0[g] = czero<cf>(); acc1[g] = czero<cf>(); }
#pragma unroll 8
  for (int c = 0; c < bs; ++c) {
    const float4 v = __ldg((const float4*)(F + (size_t)(kb + c) * n + r));
    const cf l0 = CF(v.x, v.y), l1 = CF(v.z, v.w);
#pragma unroll
    for (int g = 0; g < SGT; ++g) {
      const cf xc = Xb[c][g];
      acc0[g] = fma(l0, xc, acc0[g]);
      acc1[g] = fma(l1, xc, acc1[g]);
    }
  }
#pragma unroll
  for (int g = 0; g < SGT; ++g)
    if (g < G) {
      X[g][r] = X[g][r] - to_cd(acc0[g]);
      X[g][r + 1] = X[g][r + 1] - to_cd(acc1[g]);
    }
}

// Rows [r0, r1) of the block's column product by the threads t0.. of a
// stride: pairs of rows with 16-byte loads for complex64 factors (n even).
template <class TF, int SGT>
__device__ __forceinline__ void rows_update(const TF* __restrict__ F, int n, int r0, int r1, int kb, int bs,
                                           const TF (*Xb)[SGT], cd* const* X, int G, int t0, int stride) {
  if constexpr (std::is_same<TF, cf>::value) {
    if ((n & 1) == 0 && (r0 & 1) == 0) {
      for (int r = r0 + 2 * t0; r < r1; r += 2 * stride) {
        if (r + 1 < r1) block_row_update2<SGT>(F, n, r, kb, bs, Xb, X, G);
        else block_row_update<TF, SGT>(F, n, r, kb, bs, Xb, X, G);
      }
      return;
    }
  }
  for (int r = r0 + t0; r < r1; r += stride) block_row_update<TF, SGT>(F, n, r, kb, bs, Xb, X, G);
}

template <class TF, int SGT>
__host__ __device__ constexpr size_t solve_smem_fixed() {
  return 2 * (size_t)SB * (SB + 1) * sizeof(TF) + 2 * (size_t)SB * SGT * sizeof(TF);
}

template <class TF, bool PHYS, int SGT>
__global__ void __launch_bounds__(SolveShape<SGT>::NT) solve_blocked_kernel(
    const TF* __restrict__ LU, const int* __restrict__ piv, int n, int M, const double* __restrict__ sw,
    const cd* __restrict__ rhs, cd* __restrict__ x, int nrhs) {
  extern __shared__ __align__(16) unsigned char sraw[];
  TF (*Ls)[SB][SB + 1] = (TF (*)[SB][SB + 1])sraw;                                   // [2] diagonal blocks
  TF (*Xs)[SB][SGT] = (TF (*)[SB][SGT])(sraw + 2 * (size_t)SB * (SB + 1) * sizeof(TF));  // [2] block solutions
  int* perm = (int*)(sraw + solve_smem_fixed<TF, SGT>());  // [n] composed interchanges, then pv_s [n]
  const int m = blockIdx.x;
  const int job0 = blockIdx.y * SGT;
  const int njobs_all = (m == 0) ? nrhs : 2 * nrhs;
  if (job0 >= njobs_all) return;
  const int G = min(SGT, njobs_all - job0);
  const TF* L = LU + (size_t)m * n * n;
  const int* pv = piv + (size_t)m * n;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
  cd* X[SGT];
  for (int g = 0; g < SGT; ++g) {
    int q, ri; bool neg;
    job_of(m, M, nrhs, job0 + (g < G ? g : 0), &q, &ri, &neg);
    X[g] = x + ((size_t)q * nrhs + ri) * n;
  }
  // row interchanges (LAPACK order) composed into perm: (P b)[r] = b[perm[r]]
  int* pv_s = perm + n;  // the pivots staged in shared memory for the serial composition
  for (int r = tid; r < n; r += T) { perm[r] = r; pv_s[r] = pv[r]; }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < n; ++k) {
      int p = pv_s[k];
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
  const int nblk = (n + SB - 1) / SB;
  auto load_diag = [&](int bi, int t0, int step) {
    const int kb = bi * SB, bs = min(SB, n - kb);
    TF (*D)[SB + 1] = Ls[bi & 1];
    for (int t = t0; t < bs * bs; t += step) {
      const int r = t % bs, c = t / bs;
      D[r][c] = L[(size_t)(kb + c) * n + kb + r];
    }
  };
  // forward: L unit lower
  load_diag(0, tid, T);
  if (nblk > 1) load_diag(1, tid, T);
  __syncthreads();
  if (tid < 32) warp_triangle<TF, SGT, true>(Ls[0], Xs[0], X, 0, min(SB, n), G, lane);
  __syncthreads();
  for (int i = 0; i < nblk; ++i) {
    const int kb = i * SB, bs = min(SB, n - kb), b = i & 1;
    const int kn = kb + SB, bsn = min(SB, n - kn);
    if (tid < 64) {
      if (bsn > 0) {
        if (tid < bsn) block_row_update<TF, SGT>(L, n, kn + tid, kb, bs, Xs[b], X, G);
        asm volatile("bar.sync 1, 64;" ::: "memory");
        if (tid < 32) warp_triangle<TF, SGT, true>(Ls[b ^ 1], Xs[b ^ 1], X, kn, bsn, G, lane);
      }
    } else {
      if (i + 2 < nblk) load_diag(i + 2, tid - 64, T - 64);
      rows_update<TF, SGT>(L, n, kn + SB, n, kb, bs, Xs[b], X, G, tid - 64, T - 64);
    }
    __syncthreads();
  }
  // backward: U upper, non-unit diagonal
  const int last = nblk - 1;
  load_diag(last, tid, T);
  if (last >= 1) load_diag(last - 1, tid, T);
  __syncthreads();
  if (tid < 32) warp_triangle<TF, SGT, false>(Ls[last & 1], Xs[last & 1], X, last * SB, n - last * SB, G, lane);
  __syncthreads();
  for (int i = last; i >= 0; --i) {
    const int kb = i * SB, bs = min(SB, n - kb), b = i & 1;
    const int kp = kb - SB;  // the block above (full size)
    if (tid < 64) {
      if (i >= 1) {
        block_row_update<TF, SGT>(L, n, kp + tid, kb, bs, Xs[b], X, G);
        asm volatile("bar.sync 1, 64;" ::: "memory");
        if (tid < 32) warp_triangle<TF, SGT, false>(Ls[b ^ 1], Xs[b ^ 1], X, kp, SB, G, lane);
      }
    } else {
      if (i - 2 >= 0) load_diag(i - 2, tid - 64, T - 64);
      rows_update<TF, SGT>(L, n, 0, kp, kb, bs, Xs[b], X, G, tid - 64, T - 64);
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

// Vectors per CTA: 32 when that still leaves two CTAs per SM (many
// right-hand sides: every group reads the whole factor, so wider groups read
// it fewer times), else 8 when that leaves four, else 4 (more CTAs hide the
// latency of the per-block triangle steps; measured on the cylinder's 65
// modes x 32 vectors: 4 vectors 53 ms, 8 vectors 63 ms, 2 vectors 75 ms for
// the three correction solves with residuals, with 256 threads per CTA).
template <class TF, bool PHYS, int W>
static void launch_solve_w(const TF* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x, int nrhs,
                           int smem_perm, cudaStream_t s) {
  const int groups = (2 * nrhs + W - 1) / W;
  const int smem = (int)solve_smem_fixed<TF, W>() + smem_perm;
  smem_optin(solve_blocked_kernel<TF, PHYS, W>);
  solve_blocked_kernel<TF, PHYS, W><<<dim3(M + 1, groups), SolveShape<W>::NT, smem, s>>>(LU, piv, n, M, sw, rhs, x,
                                                                                          nrhs);
}

template <class TF, bool PHYS>
static void launch_solve_blocked(const TF* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x,
                                 int nrhs, cudaStream_t s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = 2 * n * (int)sizeof(int);
  const long long modes = M + 1;
  if (modes * ((2 * nrhs + 31) / 32) >= 2LL * sms) launch_solve_w<TF, PHYS, 32>(LU, piv, n, M, sw, rhs, x, nrhs, smem, s);
  else if (modes * ((2 * nrhs + SG - 1) / SG) >= 4LL * sms) launch_solve_w<TF, PHYS, SG>(LU, piv, n, M, sw, rhs, x, nrhs, smem, s);
  else launch_solve_w<TF, PHYS, 4>(LU, piv, n, M, sw, rhs, x, nrhs, smem, s);
}

void lu_solve_modes(const cd* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x, int nrhs,
                    cudaStream_t s) {
  launch_solve_blocked<cd, true>(LU, piv, n, M, sw, rhs, x, nrhs, s);
}

void lu_correction_solve_c64(const cf* LU, const int* piv, int n, int M, const cd* r, cd* d, int nrhs,
                             cudaStream_t s) {
  launch_solve_blocked<cf, false>(LU, piv, n, M, nullptr, r, d, nrhs, s);
}
