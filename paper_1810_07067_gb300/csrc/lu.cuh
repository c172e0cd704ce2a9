// Batched dense complex LU with partial pivoting and triangular solves.
#pragma once
#include <cuda_runtime.h>
#include "cplx.cuh"

#define LU_NB 32

// Factor `batch` column-major n x n matrices (stride n*n) in place: P A = L U.
// piv[b*n + k] = row interchanged with row k (0-based, LAPACK order);
// info[b] = 0, or k+1 for the first exactly zero pivot column k.
struct LuTiming {
  double gemm_ms = 0.0;      // summed device time of the trailing-update launches
  double gemm_flops = 0.0;   // their algorithmic flops (8 per complex multiply-add)
  int gemm_launches = 0;
  int launches = 0;          // all kernel launches of the factorization
};
void lu_factor_batched(cd* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* t = nullptr);
// The same factorization in complex64 (mixed-precision path).
// The trailing updates run on tensor cores (tcgen05, split-BF16); ws is a
// device workspace of lu_c64_workspace_bytes(n, batch) bytes (256-byte
// aligned); tc_err (device int, may be null) is set if a bounded wait gives up.
size_t lu_c64_workspace_bytes(int n, int batch);
void lu_factor_batched_c64(cf* A, int n, int batch, int* piv, int* info, cudaStream_t s, LuTiming* t, int* tc_err,
                           void* ws);

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
