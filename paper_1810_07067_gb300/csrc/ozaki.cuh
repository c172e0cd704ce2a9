// FP64-accurate complex GEMM on BF16 tensor cores (exact digit slicing), used
// for the refinement residuals of the mixed-precision path.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "cplx.cuh"

#define OZ_S 8        // digits per value (7 bits each)
#define OZ_RT 128     // output rows per CTA
#define OZ_JT 32      // right-hand sides per CTA (largest job tile; 16 when there are at most 16 jobs)
#define OZ_KT 16      // k per tile
#define OZ_CHUNK 16   // k-tiles per exact FP32 accumulation (256 values of k)

size_t ozaki_matrix_slices_elems(int npad, int batch);  // bf16 elements
// job tile (right-hand-side columns of one MMA) for nrhs right-hand sides:
// 16 when the 2 nrhs jobs (modes +m and -m) fit one tile of 16, else 32
inline int ozaki_job_tile(int nrhs) { return 2 * nrhs <= 16 ? 16 : OZ_JT; }
inline int ozaki_job_tiles(int nrhs) { const int jt = ozaki_job_tile(nrhs); return (2 * nrhs + jt - 1) / jt; }
size_t ozaki_vector_slices_elems(int npad, int batch, int njt, int jt);

// Slices of the complex matrices A[batch][n][n] (column-major) for rows padded
// to npad (multiple of 128), given rowscale[batch][npad], the power-of-two
// row scales (2^e with every |Re a|, |Im a| of the row below 2^e / 2; written
// by mixed_prepare).
void ozaki_slice_matrix(const cd* A, int n, int npad, int batch, __nv_bfloat16* Asl, const double* rowscale,
                        cudaStream_t s);

// r = b' - A'_{+-m} y for modes -M..M with the sliced matrices (see mixed.cu);
// Ysl / colscale are workspaces; err is set on a timed-out device wait.
void ozaki_residual(const __nv_bfloat16* Asl, const double* rowscale, int n, int npad, int M, const cd* bw,
                    const cd* y, cd* r, int nrhs, double* rnorm, __nv_bfloat16* Ysl, double* colscale, int* err,
                    cudaStream_t s);

// Real product Y[c * ldy + r] = sum_k A[r][k] B[k][c], c < ncols, on BF16
// tensor cores with FP64 accuracy (the digit slicing above): A as the 8
// digits of its rows (rows_pad a multiple of 128, row scales Ascale), B as
// the digits of b / bscale built on the host by ozaki_real_b_host; K =
// 16 nkt <= 272.  err is set on a timed-out device wait.
#define OZR_KMAX 272
size_t ozaki_real_a_elems(int rows_pad, int nkt);   // bf16 elements of the A digits
size_t ozaki_real_b_elems(int ncols, int nkt);      // bf16 elements of the B digits
void ozaki_real_b_host(const double* b, int K, int ncols, double bscale, int nkt, __nv_bfloat16* out);
void ozaki_real_gemm(const __nv_bfloat16* Asl, const double* Ascale, int rows_pad, const __nv_bfloat16* Bsl,
                     double bscale, int nkt, double* Y, int ldy, int ncols, int* err, cudaStream_t s);
