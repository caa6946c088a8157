// Host check of the integer-based binary64 <-> binary32 conversions against
// the C++ conversions: d2f within half a binary32 ulp (ties may differ by one
// ulp: rounding away from zero against the hardware's ties-to-even), exact
// f2d, the special values; prints "ok <n>" or the first failure.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>
#include <limits>
#include "tb_fpconv.cuh"

static int fail(const char* what, double x, float got, float want) {
  std::printf("FAIL %s x=%.17g got=%.9g want=%.9g\n", what, x, got, want);
  return 1;
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-120, 120);
  long n = 0;
  for (int i = 0; i < 2000000; ++i) {
    const double x = std::ldexp(u(rng), ex(rng));
    const float got = tbconv::d2f(x);
    float want = (float)x;
    if (std::fabs(x) < 1.1754943508222875e-38) want = std::copysign(0.f, (float)x);   // flushed
    if (got != want) {
      // only a tie may differ, by one ulp
      const float up = std::nextafter(want, std::copysign(INFINITY, want));
      const double mid = 0.5 * ((double)want + (double)up);
      if (!(got == up && x == mid) && !(got == std::nextafter(want, -std::copysign(INFINITY, want)) && x == 0.5 * ((double)want + (double)got)))
        return fail("d2f", x, got, want);
    }
    const float f = (float)x;
    if (std::fabs(f) >= std::numeric_limits<float>::min() || f == 0.f) {
      const double back = tbconv::f2d(f);
      if (back != (double)f) return fail("f2d", (double)f, (float)back, f);
    }
    ++n;
  }
  const double specials[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 1e39, -1e39,
                             1.1754943508222875e-38, 1e-40, INFINITY, -INFINITY};
  for (double x : specials) {
    const float got = tbconv::d2f(x);
    float want = (float)x;
    if (std::fabs(x) < 1.1754943508222875e-38) want = std::copysign(0.f, (float)x);   // flushed
    if (!(got == want && std::signbit(got) == std::signbit(want))) return fail("special", x, got, want);
    ++n;
  }
  if (!std::isnan(tbconv::d2f(NAN)) || !std::isnan(tbconv::f2d(NAN))) return fail("nan", NAN, 0.f, NAN);
  if (tbconv::f2d(INFINITY) != INFINITY || tbconv::f2d(-0.f) != 0.0 || !std::signbit(tbconv::f2d(-0.f)))
    return fail("f2d special", 0.0, 0.f, 0.f);
  std::printf("ok %ld\n", n);
  return 0;
}
