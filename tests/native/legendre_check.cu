// Host-side driver of the split pairs' Laplace-type coefficients
// (legendre_one in csrc/green.cu, linked from a host compile of that file).
// Reads lines "rt dr dz Mq Ms" from stdin and prints per line the Mq + 1
// coefficients P^_m and then the Ms coefficients S^_m.
#include <cstdio>
#include <vector>
#include "green.cuh"

// the library's error hook (defined with the C ABI, not linked here)
void mueller_internal_set_error(const char*) {}

int main() {
  double rt, dr, dz;
  int Mq, Ms;
  while (scanf("%lf %lf %lf %d %d", &rt, &dr, &dz, &Mq, &Ms) == 5) {
    std::vector<double> leg((size_t)(Mq + 1) + Ms);
    legendre_one(rt, dr, dz, 0, 1, Mq, Ms, leg.data(), nullptr, 0);
    for (double v : leg) printf("%.17g ", v);
    printf("\n");
  }
  return 0;
}
