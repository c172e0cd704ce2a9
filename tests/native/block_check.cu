// Host-side driver of the Mueller 4 x 4 block arithmetic of the far-pair
// assembly (csrc/block.cuh), compiled for the CPU: reads cases from stdin
// and prints, per case, the block of mueller_block_spec<false> and of the
// specialised mueller_block_spec<true> (the general block again when the
// case is not eligible), 32 complex numbers as "re im" lines.
//
// Case layout (whitespace separated): formulation omega, k0 k1 eps0 mu0 eps1
// mu1 (complex: re im each), M m rt rpt zpt rs rps zps, then the spectra
// S[f][mode], f < 9, mode < M + 2 (complex).  Unit quadrature weight: the
// block's three weights are rs r's, rs and rs z's.
#include <cstdio>
#include <vector>
#include "../../paper_1810_07067_gb300/csrc/block.cuh"

static cd rd_c() {
  double a = 0, b = 0;
  if (scanf("%lf %lf", &a, &b) != 2) return C(0.0);
  return C(a, b);
}

int main() {
  int ncase = 0;
  if (scanf("%d", &ncase) != 1) return 2;
  for (int q = 0; q < ncase; ++q) {
    int form = 0, M = 0, m = 0;
    double omega = 0, rt, rpt, zpt, rs, rps, zps;
    if (scanf("%d %lf", &form, &omega) != 2) return 2;
    const cd k0 = rd_c(), k1 = rd_c(), eps0 = rd_c(), mu0 = rd_c(), eps1 = rd_c(), mu1 = rd_c();
    if (scanf("%d %d %lf %lf %lf %lf %lf %lf", &M, &m, &rt, &rpt, &zpt, &rs, &rps, &zps) != 8) return 2;
    const int Ms = M + 2;
    std::vector<cd> S(9 * Ms);
    for (auto& v : S) v = rd_c();
    // the block coefficients as the library's set-up forms them
    const cd iw = C(0.0, omega);
    AsmParams ap{};
    ap.k0sq = k0 * k0;
    ap.k1sq = k1 * k1;
    if (form == 0) {
      ap.aEJ = C(1.0); ap.aHM = C(-1.0);
      ap.cEM0 = -(iw * eps0); ap.cEM1 = iw * eps1;
      ap.cHJ0 = -(iw * mu0); ap.cHJ1 = iw * mu1;
    } else {
      ap.aEJ = mu0 / eps0; ap.aHM = -(eps0 / mu0);
      ap.cEM0 = -(iw * mu0); ap.cEM1 = iw * mu1;
      ap.cHJ0 = -(iw * eps0); ap.cHJ1 = iw * eps1;
    }
    ap.simple = ap.k0sq.y == 0.0 && ap.k1sq.y == 0.0 && ap.cEM0.x == 0.0 && ap.cEM1.x == 0.0 && ap.cHJ0.x == 0.0 &&
                ap.cHJ1.x == 0.0 && ap.aEJ.x == 1.0 && ap.aEJ.y == 0.0 && ap.aHM.x == -1.0 && ap.aHM.y == 0.0;
    const double fac[3] = {rs * rps, rs, rs * zps};
    cd g[4][4], s[4][4];
    mueller_block_spec<false>(S.data(), Ms, 0, fac, m, ap, rt, 1.0 / rt, rpt, zpt, g);
    if (ap.simple) mueller_block_spec<true>(S.data(), Ms, 0, fac, m, ap, rt, 1.0 / rt, rpt, zpt, s);
    else mueller_block_spec<false>(S.data(), Ms, 0, fac, m, ap, rt, 1.0 / rt, rpt, zpt, s);
    printf("%d\n", ap.simple);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) printf("%.17g %.17g\n", g[a][b].x, g[a][b].y);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) printf("%.17g %.17g\n", s[a][b].x, s[a][b].y);
  }
  return 0;
}
