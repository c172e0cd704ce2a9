// Host-side check of the integer rounding used by the sampling kernels'
// digit rows (digits.cuh): fixed_rn(v, S) must equal round(v 2^S) with ties
// to even -- the C library's llrint of the exact product ldexp(v, S) in the
// default rounding mode -- for every |v 2^S| < 2^55, including exact ties,
// subnormal samples and rows whose scale is subnormal; abs_bits must order
// finite values as fabs does; digits28 must split each fixed-point value
// into 8 balanced base-128 digits that sum back to it.  Exit status 0 when
// every case agrees.
#include <cmath>
#include <cstdio>
#include <random>
#include "../../paper_1810_07067_gb300/csrc/digits.cuh"

int main() {
  std::mt19937_64 gen(1810);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  long long n = 0, bad = 0;
  auto check = [&](double v, int S) {
    const long long ref = llrint(ldexp(v, S));
    const long long got = fixed_rn(v, S);
    ++n;
    if (ref != got) {
      if (bad < 5) printf("fixed_rn(%.17g, %d) = %lld, round-to-nearest-even gives %lld\n", v, S, got, ref);
      ++bad;
    }
  };
  // samples of a row with scale 2^E (|v| < 2^(E-1)), S = 56 - E, and values far below the row's largest
  for (int it = 0; it < 2000000; ++it) {
    const int E = (int)(gen() % 200) - 100;
    const double v = ldexp(U(gen) * ldexp(0.5, E), -(int)(gen() % 80));
    check(v, 56 - E);
  }
  // exact ties k + 1/2 and quarter points at several scales
  for (long long k = -3000; k <= 3000; ++k)
    for (int E = -40; E <= 40; E += 8) {
      check(ldexp((double)k + 0.5, E - 56), 56 - E);
      check(ldexp((double)k + 0.25, E - 56), 56 - E);
      check(ldexp((double)k + 0.75, E - 56), 56 - E);
    }
  // the top of the range, zeros, subnormal samples and subnormal row scales
  for (int it = 0; it < 200000; ++it) {
    check(U(gen) * 0.4999999999, 56);
    check(ldexp(U(gen), -1074 + 50), 1074 - 10);
  }
  check(0.0, 56);
  check(-0.0, 56);
  check(4.9406564584124654e-324, 1074);
  check(-4.9406564584124654e-324, 1073);
  check(ldexp(3.0, -1074), 1094);
  check(ldexp(1.0, -1022), 1032);
  long long order_bad = 0;
  for (int it = 0; it < 200000; ++it) {
    const double a = ldexp(U(gen), (int)(gen() % 400) - 200), b = ldexp(U(gen), (int)(gen() % 400) - 200);
    if ((fabs(a) < fabs(b)) != (abs_bits(a) < abs_bits(b))) ++order_bad;
  }
  // digits28: balanced base-128 digits of F = round(v 2^56), |v| < 1/2, that
  // sum back to F exactly, each exact in BF16 (|d| <= 64, the top one too)
  long long digit_bad = 0;
  auto check_digits = [&](long long F) {
    int d[OZ_S];
    digits28(F, d);
    long long back = 0;
    bool in_range = true;
    for (int s = 0; s < OZ_S; ++s) {
      back = back * 128 + d[s];
      in_range = in_range && d[s] >= -64 && d[s] <= 64;
    }
    if (back != F || !in_range) {
      if (digit_bad < 5) printf("digits28(%lld) does not sum back or leaves [-64, 64]\n", F);
      ++digit_bad;
    }
  };
  for (int it = 0; it < 2000000; ++it) check_digits(fixed_rn(U(gen) * 0.5, 56));
  const long long edge = (1ll << 55) - 1;
  for (long long F : {0ll, 1ll, -1ll, 63ll, 64ll, 65ll, -64ll, -65ll, edge, -edge, edge - 64, -(edge - 64)})
    check_digits(F);
  printf("%lld rounding cases, %lld mismatches; %lld ordering mismatches; %lld digit mismatches\n", n, bad,
         order_bad, digit_bad);
  return (bad || order_bad || digit_bad) ? 1 : 0;
}
