// Host-side check of the B operand of the tensor-core transform over phi
// (ozaki_real_b_host in csrc/ozaki.cu, linked from a host compile): for the
// cosine matrices b(j, m) = cos(2 pi m j / n) of grids n = 16 .. 512 and
// ncols modes, the 8 balanced base-128 digits stored for b / 2 at the
// operand layout (column tile of 32, k-tile of 16, digit-major, 8 x 8 core
// matrices) must sum back to round(b / 2 * 2^56) / 2^56, every digit within
// [-64, 64], and every element outside the matrix zero.  Prints the largest
// reconstruction error in units of 2^-56 and the number of violations.
#include <cmath>
#include <cstdio>
#include <vector>
#include <cuda_bf16.h>
#include "ozaki.cuh"

int main() {
  long long bad = 0, checked = 0;
  double worst = 0.0;
  const int nt = 32, kt = 16, nd = 8;
  for (int n = 16; n <= 512; n += 8)
    for (int ncols : {n / 2 + 1 < 130 ? n / 2 + 1 : 130, 12}) {
      const int K = n / 2 + 1, nkt = (K + 15) / 16;
      if (ncols > K) continue;
      std::vector<double> b((size_t)K * ncols);
      for (int j = 0; j < K; ++j)
        for (int m = 0; m < ncols; ++m) b[(size_t)j * ncols + m] = std::cos(2.0 * M_PI * (double)((long long)m * j % n) / n);
      std::vector<__nv_bfloat16> out(ozaki_real_b_elems(ncols, nkt));
      ozaki_real_b_host(b.data(), K, ncols, 2.0, nkt, out.data());
      const int ntile = (ncols + nt - 1) / nt;
      for (int t = 0; t < ntile; ++t)
        for (int q = 0; q < nkt; ++q)
          for (int cc = 0; cc < nt; ++cc)
            for (int kk = 0; kk < kt; ++kk) {
              const int c = t * nt + cc, k = q * kt + kk;
              const int off = ((cc >> 3) * 2 + (kk >> 3)) * 64 + (cc & 7) * 8 + (kk & 7);
              long long F = 0;
              bool range_ok = true;
              for (int s = 0; s < nd; ++s) {
                const float d = __bfloat162float(out[((size_t)t * nkt + q) * (nd * nt * kt) + (size_t)s * nt * kt + off]);
                range_ok = range_ok && d >= -64.f && d <= 64.f && d == std::floor(d);
                F = F * 128 + (long long)d;
              }
              ++checked;
              if (c >= ncols || k >= K) {
                if (F != 0 || !range_ok) ++bad;
                continue;
              }
              const double want = std::ldexp(b[(size_t)k * ncols + c] / 2.0, 56);
              const double err = std::fabs((double)F - want);
              if (err > worst) worst = err;
              if (err > 0.5 || !range_ok) ++bad;
            }
    }
  printf("%lld elements, largest error %.3g (units of 2^-56), %lld violations\n", checked, worst, bad);
  return bad ? 1 : 0;
}
