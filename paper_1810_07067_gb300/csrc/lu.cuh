// Batched dense complex LU with partial pivoting and triangular solves.
#pragma once
#include <cuda_runtime.h>
#include "cplx.cuh"

#define LU_NB 32

// Factor `batch` column-major n x n matrices (stride n*n) in place: P A = L U.
// piv[b*n + k] = row interchanged with row k (0-based, LAPACK order);
// info[b] = 0, or k+1 for the first exactly zero pivot column k.
struct LuTiming {
  double gemm_ms = 0.0;      // summed device time of the trailing-update launches (0 when graph-launched)
  double gemm_flops = 0.0;   // their algorithmic flops (8 per complex multiply-add)
  double gemm_bytes = 0.0;   // the trailing matrices' bytes, read and written once per update
  int gemm_launches = 0;     // steps with a trailing update
  int launches = 0;          // all kernel launches of the factorization
  int graph = 0;             // 1: the steps ran as one captured CUDA graph
  int tile_steps[3] = {0, 0, 0};  // complex64: steps whose update used column tiles of 32, 64, 128
};
void lu_factor_batched(cd* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* t = nullptr);
// The same factorization in complex64 (mixed-precision path).
// The trailing updates run on tensor cores (tcgen05, split-BF16); ws is a
// device workspace of lu_c64_workspace_bytes(n, batch) bytes (256-byte
// aligned); tc_err (device int, may be null) is set if a bounded wait gives up.
// tile: column tile of the update (32, 64 or 128), 0 = autotuned per step.
size_t lu_c64_workspace_bytes(int n, int batch);
void lu_factor_batched_c64(cf* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* t, int* tc_err,
                           void* ws, int tile = 0);

// One matrix of a (possibly ragged) batched factorization: A is n x n
// column-major (complex128 or complex64), piv [n], info [1]; ws (complex64
// only) is its own lu_c64_workspace_bytes(n, 1)-byte workspace, 16-byte
// aligned.
struct LuMat {
  void* A;
  int* piv;
  int* info;
  void* ws;
  int n;
  int pad_;
};
// Factor all `count` matrices (any mix of sizes) with one launch per kernel
// and step over all of them; with graph = true the whole step sequence is
// captured into a CUDA graph and launched once on s.  Returns the first CUDA
// error (cudaSuccess when every launch was issued).
cudaError_t lu_factor_many(const LuMat* items, int count, bool c64, cudaStream_t s, LuTiming* t, int* tc_err,
                           int tile, bool graph);
// The autotuner's decisions so far: per entry the upper end of its trailing-size
// bucket, of its matrix-count bucket, the tile chosen and the measured ms per
// matrix of tiles 32, 64, 128 (ms[3k..3k+2]); returns the number of entries.
int lu_tile_table(int* rest_hi, int* count_hi, int* tile, float* ms, int cap);

// Solve with factors of modes m = 0..M for right-hand sides of modes -M..M:
// rhs/x layout [2M+1][nrhs][n] (mode q = m + M); sw[n/4] = sqrt of the L2 weights of the nodes
// (rows scaled by sw, unknowns by 1/sw inside the factors); negative modes use
// the reflection A_{-m} = D_r A_m D_c with D_r = (-1,1,1,-1), D_c = (1,-1,-1,1)
// per node.
void lu_solve_modes(const cd* LU, const int* piv, int n, int M, const double* sw, const cd* rhs, cd* x, int nrhs,
                    cudaStream_t s);

// Mixed path: d = A'^{-1} r with the complex64 factors of modes 0..M in FP32
// arithmetic, in the L2-weighted space (no sqrt-weight scaling), for all modes
// -M..M (layout [2M+1][nrhs][n], -m by reflection).
void lu_correction_solve_c64(const cf* LU, const int* piv, int n, int M, const cd* r, cd* d, int nrhs,
                             cudaStream_t s);

// Held by a thread while it captures the LU's launches into a CUDA graph;
// code that frees device memory (and so synchronizes the device) takes it
// first, so that it never ends another thread's capture.
#include <mutex>
std::mutex& lu_capture_mutex();
