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
