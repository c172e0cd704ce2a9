// Per-pair azimuthal grid and highest mode of the far pairs (host and
// device; the grid ladder's tables are built on the host).
#pragma once
#include <cmath>
#include "cplx.cuh"
#include "green.cuh"

// The pair is the target (rt, zt) and the displacement (dr0, zd) = target - source.
// Split pairs are sampled on the full n_phi grid and keep all modes 0..M+1.
// A non-split pair's spectra decay like zeta^(m - K) past the band of the
// oscillating factor exp(i k rho) (zeta = chi - sqrt(chi^2 - 1), the
// singularity of 1/rho at cos phi = chi; the band is about |k| sqrt(r_t r_s):
// the phase k rho(phi) turns at most at that rate; margin K = |k|max
// sqrt(r_t r_s) + 4, whose exact tails at mode mc + 1 measured below 1e-20 of
// each family's largest coefficient in 40-digit quadrature).  So
//  - modes above mc = min(M + 1, ceil(K + ln(1/eps) / ln(1/zeta))) are below
//    eps of the family's largest coefficient and are set to zero;
//  - on an n-point grid, mode m <= mc picks up the aliases of modes n - m and
//    beyond, below eps once n >= mc + K + ln(1/eps) / ln(1/zeta);
// and the pair is sampled on the smallest grid of the ladder (every multiple
// of 8 below n_phi: two folds) that keeps modes 0..mc distinct (n >= 2 mc + 2)
// and the aliases below eps, or on the full grid when none does.  eps is the
// splitting threshold.  Neither choice changes the computed quantity by more
// than eps of a family's largest coefficient.  The cosine transform folds
// samples j and n/2 - j (cos of the mirrored angle is (-1)^m times the
// original), halving its work.
struct PairGrid {
  int nl;        // grid size
  int mc;        // highest mode computed (modes above are zero)
  const double* cosL;  // cos(2 pi t / nl), t < nl
  const double* s2L;   // sin^2(pi j / nl), j <= nl / 2
};

__host__ __device__ __forceinline__ PairGrid full_grid(const GreenParams& gp, const double* cosT, const double* s2T) {
  return PairGrid{gp.nphi, gp.Ms - 1, cosT, s2T};
}

__host__ __device__ inline PairGrid pair_grid(const GreenParams& gp, double rt, double dr0, double zd, bool split,
                                             double lneps, const double* cosT, const double* s2T, const double* ladC,
                                             const double* ladS) {
  if (split || gp.qmax < 2) return full_grid(gp, cosT, s2T);
  const double d2 = dr0 * dr0 + zd * zd, B = 2.0 * rt * (rt - dr0);
  const double c = d2 / B;
  const double lz = log1p(c + sqrt(c * (2.0 + c)));
  const double kmax = fmax(cabs(gp.kp0.k), cabs(gp.kp1.k));
  const double K = kmax * sqrt(0.5 * B) + 4.0;
  const double span = lneps / lz;
  const int mc = (int)fmin((double)(gp.Ms - 1), ceil(K + span));
  const double need = fmax(2.0 * mc + 2.0, fmax(16.0, ceil(mc + K + span)));
  const int q = (int)ceil(need / 8.0);
  if (q > gp.qmax) return full_grid(gp, cosT, s2T);
  // ladder tables: sizes 8q' for q' = 2..qmax, cos tables then s2 tables
  const int offc = 4 * (q - 1) * q - 8, offs = 2 * (q - 1) * q - 4 + (q - 2);
  return PairGrid{8 * q, mc, ladC + offc, ladS + offs};
}
