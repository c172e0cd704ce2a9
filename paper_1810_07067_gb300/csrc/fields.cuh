#pragma once
#include <cuda_runtime.h>
#include "cplx.cuh"

struct FieldGeom {
  const double *r, *z, *rp, *zp, *w;  // nodes [N]
  int N;
};

// Modal plane-wave data: rhs[q][w][4N], q = m + M.
void launch_rhs_planewave(const FieldGeom& g, int M, cd k0, double omega, cd mu0, cd sE, cd sH,
                          const double* dirs_dev, const double* pols_dev, int nrhs, int n_theta, cd* rhs,
                          cudaStream_t s);

// Far field E[rhs][dir][3] from currents x[q][rhs][4N]; ring work buffer
// cur[rhs][N][n_theta][4].
void launch_far_field(const FieldGeom& g, int M, cd k0, double omega, cd eps0, const cd* x, int nrhs,
                      const double* dirs_dev, int ndir, int n_theta, cd* cur, cd* E, cudaStream_t s);

// Modal data from sampled incident fields EH[rhs][N][n_theta][6] (device).
void launch_rhs_samples(const FieldGeom& g, int M, cd sE, cd sH, const cd* EH, int nrhs, int n_theta, cd* rhs,
                        cudaStream_t s);

// E, H at points X[nt][3] (device) into out[rhs][nt][6]; cur is a ring work
// buffer [rhs][N][n_theta][4]; k and the four constants are the region's.
void launch_near_field(const FieldGeom& g, int M, const cd* x, int nrhs, const double* X_dev, int nt, int n_theta,
                       cd k, cd cJ, cd cM, cd dM, cd dJ, cd* cur, cd* out, cudaStream_t s);

// Far field on the grid theta_p = (p + 1/2) pi / n_polar, phi_s = 2 pi s / n_azim:
// E[rhs][p][s][3]; work buffers coef [n_polar][N][2M+3], F [rhs][n_polar][2M+1][3].
void launch_far_field_grid(const FieldGeom& g, int M, cd k0, double omega, cd eps0, const cd* x, int nrhs,
                           int n_polar, int n_azim, int n_alpha, cd* coef, cd* F, cd* E, cudaStream_t s);

// Currents x[v][n] at the nodes -> xs[v][4 nsub] at refined nodes (rows Lm[nsub][16]
// of the panel interpolants, node0 = first node of each sub-node's panel).
void launch_interp_currents(const cd* x, int n, int nsub, const int* node0, const double* Lm, long long nvec, cd* xs,
                            cudaStream_t s);
