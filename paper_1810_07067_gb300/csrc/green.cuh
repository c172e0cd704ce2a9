// Modal Green's function evaluation and per-mode assembly (Sections 3-5).
#pragma once
#include <cuda_bf16.h>
#include "cplx.cuh"
#include "special.cuh"

#define NFAM 9          // spectra per pair (see green.cu)
#define P_NODES 16      // nodes per panel

struct GreenParams {
  int M;       // modes 0..M assembled (negative modes follow by reflection)
  int Ms;      // M + 2 spectral coefficients per family (m = 0..M+1)
  int nphi;    // azimuthal samples on [0, 2pi)
  int H;       // nphi/2 + 1 samples on [0, pi]
  int Mq;      // nphi/2 - 1: bandwidth of the Laplace coefficients
  int qmax;    // grid ladder for non-split pairs: sizes 8q, q = 2..qmax (8 qmax < nphi; 0: none)
  KPow kp0, kp1;
  cd gamma0;   // -(k0^2 - k1^2)/4
  int k0_real, k1_real;  // real wavenumbers take the real-arithmetic path
};

// Block coefficients of eq. mullerrep / eq. dualmullrep.
struct AsmParams {
  cd k0sq, k1sq;
  cd aEJ, aHM;          // K-block factors
  cd cEM0, cEM1;        // E rows, M columns: cEM0 N0 + cEM1 N1
  cd cHJ0, cHJ1;        // H rows, J columns
  cd dEM, dHJ;          // identity terms
  int simple;           // 1: k0^2, k1^2 real, cEM and cHJ purely imaginary, aEJ = 1, aHM = -1
};

struct NodeGeom {
  const double *r, *z, *rp, *zp, *w, *sw;  // [N]; sw = sqrt(w)
};

struct SupportTable {
  const double *r, *z, *rp, *zp, *W;  // support points, [n_panels * PTS_PER_PANEL]
  const double *dr, *dz;              // target - point displacement (own-panel points)
  const double* Lself;                // [16][SELF_PTS][16]
  const double* Ladj;                 // [2 rules][2 ends][ADJ_PTS][16]  (rule 0 smooth junction, 1 corner;
                                      // end 0: shared end -1, 1: shared end +1)
  const int* adj_rule;                // [n_panels][2] rule of each panel end (-1: no neighbour)
  const int* adj_n;                   // [n_panels][2] its number of points (0: no neighbour)
};

#include "mueller_near_rules.h"
// support points of the near-panel rules (Section 5): the target's own panel
// takes the generalized Gaussian rule on each side of the target, each
// neighbouring panel the compressed generalized Gaussian rule for smooth
// junctions (both tables of mueller_near_rules.h) or, at a corner, a graded
// composite rule of 96 points; ADJ_PTS slots are reserved per panel end
#define SELF_SIDE MUELLER_SELF_SIDE
#define SELF_PTS (2 * SELF_SIDE)
#define ADJ_PTS 96
#define NEAR_MAX_PTS (SELF_PTS > ADJ_PTS ? SELF_PTS : ADJ_PTS)  // the largest rule
#define PTS_PER_PANEL (P_NODES * SELF_PTS + 2 * ADJ_PTS)
#define NEAR_SLOTS (SELF_PTS + 2 * ADJ_PTS)   // support points per target

struct BuildArgs {
  GreenParams gp;
  AsmParams ap;
  NodeGeom geo;
  SupportTable sup;
  int N, n_panels, closed;
  const double* cosT;   // [nphi] cos(2 pi t / nphi)
  const double* s2T;    // [H] sin^2(pi j / nphi)
  const double* ladC;   // grid ladder: cos(2 pi t / 8q), t < 8q, for q = 2..qmax, concatenated
  const double* ladS;   // sin^2(pi j / 8q), j <= 4q, for q = 2..qmax, concatenated
  const int* split_far; // [N*N] split id or -1 (far-panel pairs)
  const int* split_sup; // [N*NEAR_SLOTS] split id or -1
  const double* leg;    // Legendre scratch: [(Mq+1) + Ms][n_split] (index-major)
                        // split pairs are given as (r_t, z_t, r_t - r_s, z_t - z_s)
  long long n_split;
  cd* spec_sup;         // [N*NEAR_SLOTS][NFAM][Ms] support spectra scratch
  cd* A;                // [M+1][n][n] column-major per mode
  int kc;               // columns per CTA in the near contraction
  double lneps;         // -ln(split threshold): grid decimation criterion
  int tq;               // far_kernel tail queue: pairs per flush (0 = none, see far_tail_pairs)
  cd* tailq;            // its spectra scratch (far_tail_scratch elements)
  int* tailij;          // its (target, source) scratch
};

// shared memory used by one warp of the pair-spectra routine (16-byte multiple)
HD int green_smem_bytes(const GreenParams& gp) {
  int b = (NFAM * gp.H + NFAM * gp.Ms) * 16 + (gp.H + gp.Mq + 1) * 8;
  return (b + 15) & ~15;
}

// Laplace-type coefficients of one split pair p (target r_t, displacement dr, dz)
// into leg (stride n, rows 0..Mq P^_m, rows Mq+1.. S^_m).
__host__ __device__ void legendre_one(double rt, double dr, double dz, long long p, long long n, int Mq, int Ms,
                                      double* leg, const double* rinv, int nr);

// host-side launchers (green.cu)
void launch_legendre(const double* pairs, long long n_split, int Mq, int Ms, double* leg, cudaStream_t s);
int far_tail_pairs(const GreenParams& gp);
// elements of BuildArgs::tailq (return) and tailij (*ij_elems) for the launch of launch_far_assembly
size_t far_tail_scratch(const BuildArgs& a, size_t* ij_elems);
void launch_far_assembly(const BuildArgs& a, cudaStream_t s);
void launch_support_spectra(const BuildArgs& a, cudaStream_t s);
// support spectra with the transform on the tensor cores, for the support
// pairs list[q0 .. q0 + count) (p = target * NEAR_SLOTS + slot): samples ->
// row digits (rows = 18 per pair, a multiple of 128 padded) -> (ozaki_real_gemm) ->
// spectra into BuildArgs::spec_sup
void launch_support_samples(const BuildArgs& a, const int* list, int q0, int count, __nv_bfloat16* Asl,
                            double* Ascale, int nkt, cudaStream_t s);
void launch_support_post(const BuildArgs& a, const int* list, int q0, int count, const double* Y, int ldy,
                         cudaStream_t s);
// far pairs with the transform on the tensor cores: bins by grid size
// (g.nl / 8), a bin-sorted pair list, then per bin and chunk the samples'
// digit rows, ozaki_real_gemm with the bin's cos(2 pi m j / nl), and the
// blocks (the same modes, zeros and tail queue as far_kernel)
void launch_far_bins(const BuildArgs& a, unsigned short* bin_of, int* counts, cudaStream_t s);
void launch_far_scatter(long long total, const unsigned short* bin_of, int* cursor, int* list, cudaStream_t s);
void launch_far_samples(const BuildArgs& a, const int* list, int q0, int count, __nv_bfloat16* Asl, double* Ascale,
                        int nkt, int nl, cudaStream_t s);
void launch_far_assemble(const BuildArgs& a, const int* list, int q0, int count, const double* Y, int ldy, int ncols,
                         int nl, cudaStream_t s);
void launch_near_assembly(const BuildArgs& a, cudaStream_t s);
void launch_pair_spectra(const GreenParams& gp, const double* pairs, const int* split_id, const double* leg,
                         long long n_split, long long npairs, const double* cosT, const double* s2T,
                         cd* out, cudaStream_t s);
void upload_series_tables(const SeriesTables& t);
int green_smem_per_warp(const GreenParams& gp);
// whether one warp's shared memory (green_smem_bytes) fits the device's per-CTA opt-in limit
bool green_fits_smem(const GreenParams& gp);
