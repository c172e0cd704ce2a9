// Host-side driver of the special functions of the split modal kernels
// (csrc/special.cuh), compiled for the CPU.  Reads lines from stdin:
//   0 kre kim su   -> entire(k, su), seven complex values C S Gam Gam2 Gamp Sp Spp
//   1 k su         -> entire_real(k, su), the same seven values
//   2 kp           -> ellipk_c(kp)
//   3 x y z        -> carlson_rd(x, y, z)
// and prints one line of results per input line ("re im" pairs or a real).
#include <cstdio>
#include "../../paper_1810_07067_gb300/csrc/special.cuh"

static void put(const Ent& e) {
  const cd v[7] = {e.C, e.S, e.Gam, e.Gam2, e.Gamp, e.Sp, e.Spp};
  for (int q = 0; q < 7; ++q) printf("%.17g %.17g ", v[q].x, v[q].y);
  printf("\n");
}

int main() {
  SeriesTables T;
  fill_series_tables(&T);
  int kind;
  while (scanf("%d", &kind) == 1) {
    if (kind == 0) {
      double kr, ki, su;
      if (scanf("%lf %lf %lf", &kr, &ki, &su) != 3) return 2;
      put(entire(T, kpow(C(kr, ki)), su));
    } else if (kind == 1) {
      double k, su;
      if (scanf("%lf %lf", &k, &su) != 2) return 2;
      put(entire_real(T, k, su));
    } else if (kind == 2) {
      double kp;
      if (scanf("%lf", &kp) != 1) return 2;
      printf("%.17g\n", ellipk_c(kp));
    } else if (kind == 3) {
      double x, y, z;
      if (scanf("%lf %lf %lf", &x, &y, &z) != 3) return 2;
      printf("%.17g\n", carlson_rd(x, y, z));
    } else {
      return 2;
    }
  }
  return 0;
}
