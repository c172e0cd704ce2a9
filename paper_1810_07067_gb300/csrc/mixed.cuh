// Mixed-precision path: complex64 factors, FP64 residuals, iterative refinement.
#pragma once
#include <cuda_runtime.h>
#include "cplx.cuh"

// One pass over `batch` column-major n x n matrices: A32 = complex64 copy (skipped when A32 is null),
// normA[b] = infinity norm of matrix b and, when rowscale is not null, the
// power-of-two row scales of the tensor-core residuals for rows 0..npad-1
// (rowscale[b * npad + i]; see ozaki_slice_matrix).
void mixed_prepare(const cd* A, int n, int batch, cf* A32, double* normA, double* rowscale, int npad, cudaStream_t s);
// bw = S b (physical -> weighted), infinity norm per vector into bnorm
void mixed_scale(const cd* b, cd* bw, const double* sw, int n, long long nvec, double* bnorm, cudaStream_t s);
// r = bw - A'_{+-m} y for all modes -M..M ([2M+1][nrhs][n]); infinity norm per vector into rnorm
void mixed_residual(const cd* A, int n, int M, const cd* bw, const cd* y, cd* r, int nrhs, double* rnorm,
                    cudaStream_t s);
// y += d (or y = d when first), infinity norm per vector into ynorm
void mixed_update(cd* y, const cd* d, int n, long long nvec, bool first, double* ynorm, cudaStream_t s);
// x = S^{-1} y
void mixed_unscale(const cd* y, cd* x, const double* sw, int n, long long nvec, cudaStream_t s);
