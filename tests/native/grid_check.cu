// Host-side driver of the far pairs' grid choice (csrc/grid.cuh, compiled
// for the CPU).  Reads lines "k0re k0im k1re k1im M nphi split_eps rt dr0 zd
// split" from stdin and prints "nl mc" per line: the grid size and the
// highest mode that pair_grid gives the pair (the full grid and M + 1 for
// split pairs or when no grid of the ladder suffices).
#include <cstdio>
#include <cmath>
#include "../../paper_1810_07067_gb300/csrc/grid.cuh"

int main() {
  double k0r, k0i, k1r, k1i, eps, rt, dr0, zd;
  int M, nphi, split;
  while (scanf("%lf %lf %lf %lf %d %d %lf %lf %lf %lf %d", &k0r, &k0i, &k1r, &k1i, &M, &nphi, &eps, &rt, &dr0, &zd,
               &split) == 11) {
    // the build's parameters of the transform over phi
    GreenParams gp{};
    gp.M = M; gp.Ms = M + 2; gp.nphi = nphi; gp.H = nphi / 2 + 1; gp.Mq = nphi / 2 - 1;
    gp.kp0 = kpow(C(k0r, k0i)); gp.kp1 = kpow(C(k1r, k1i));
    gp.qmax = (nphi - 1) / 8;
    static double dummy[1 << 16];
    const PairGrid g = pair_grid(gp, rt, dr0, zd, split != 0, -std::log(eps), dummy, dummy, dummy, dummy);
    printf("%d %d\n", g.nl, g.mc);
  }
  return 0;
}
