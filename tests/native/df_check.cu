// Host check of the double-float transformations the outer Krylov kernels use
// (paper_1712_06091_gb300/csrc/df.cuh, compiled here for the host):
//   two-sum: s + e equals a + b exactly;
//   the FMA two-product inside df_add_prod2: a running sum of products of
//   float pairs stays within a small multiple of 2^-46 of the exact sum's
//   magnitude scale (exact reference in long double from the same pairs);
//   df_split: |v - hi - lo| <= 2^-48 |v|;
//   df_pair: hi is the float32 rounding of s + t and hi + lo equals s + t.
// Prints "ok" or the first failure.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "../../paper_1712_06091_gb300/csrc/df.cuh"

using adr::DfSum;

static int fail(const char* what, double a, double b) {
  std::printf("%s: %.17g %.17g\n", what, a, b);
  return 1;
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> mant(1.0, 2.0);
  std::uniform_int_distribution<int> ex(-20, 20), sg(0, 1);
  auto rnd = [&](int spread) {   // a float with a random sign, mantissa and exponent within +-spread
    std::uniform_int_distribution<int> e(-spread, spread);
    const double v = std::ldexp(mant(rng), e(rng));
    return (float)(sg(rng) ? -v : v);
  };

  // two-sum: exact (exponents within 28 of each other, so a + b is exact in double)
  for (int it = 0; it < 200000; ++it) {
    const float a = rnd(14), b = rnd(14);
    float s, e;
    adr::two_sum(a, b, s, e);
    if ((double)s + (double)e != (double)a + (double)b) return fail("two_sum", (double)s + e, (double)a + b);
    if (s != (float)((double)a + (double)b)) return fail("two_sum rounding", s, (double)a + b);
  }

  // df_split and df_pair
  for (int it = 0; it < 200000; ++it) {
    const double v = std::ldexp(mant(rng), ex(rng)) * (sg(rng) ? -1.0 : 1.0);
    const float2 p = adr::df_split(v);
    if (std::fabs(v - (double)p.x - (double)p.y) > std::ldexp(std::fabs(v), -48))
      return fail("df_split", v, (double)p.x + p.y);
    DfSum d{p.x, p.y};
    const float2 q = adr::df_pair(d);
    if ((double)q.x + (double)q.y != (double)p.x + (double)p.y) return fail("df_pair sum", q.x + (double)q.y, v);
    if (q.x != (float)((double)p.x + (double)p.y)) return fail("df_pair rounding", q.x, v);
  }

  // running sums of double-float products (the Gram-Schmidt dots): 256 terms,
  // signs mixed so that the sum cancels; the error bound is relative to the
  // sum of the terms' magnitudes (what the transformations guarantee)
  for (int trial = 0; trial < 2000; ++trial) {
    DfSum acc{0.f, 0.f};
    long double exact = 0.0L, scale = 0.0L;
    for (int i = 0; i < 256; ++i) {
      const double x = std::ldexp(mant(rng), ex(rng) / 4) * (sg(rng) ? -1.0 : 1.0);
      const double y = std::ldexp(mant(rng), ex(rng) / 4) * (sg(rng) ? -1.0 : 1.0);
      const float2 xs = adr::df_split(x), ys = adr::df_split(y);
      adr::df_add_prod2(acc, xs.x, xs.y, ys.x, ys.y);
      const long double xv = (long double)xs.x + xs.y, yv = (long double)ys.x + ys.y;
      exact += xv * yv;
      scale += std::fabs((double)(xv * yv));
    }
    const long double got = (long double)adr::df_double(acc);
    if (std::fabs((double)(got - exact)) > 256.0 * std::ldexp((double)scale, -46))
      return fail("df_add_prod2 sum", (double)got, (double)exact);
  }
  std::printf("ok\n");
  return 0;
}
