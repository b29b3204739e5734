// Host check of the FP64 <-> double-float conversions of dfloat.cuh (the
// integer-pipe routes the transform passes use on the GPU, compiled here for
// the host): for random values with binary exponents in [-74, 126] (the range
// of full precision), x = hi + lo to 2^-47 relative, |lo| <= ulp(hi), signs
// kept, zeros exact; for normal FP32 magnitudes below 2^-74 (float64 route, lo
// may be subnormal) at least FP32 precision; float -> double on the bit pattern equal to the cast. Prints
// the worst relative error of the full-precision range and the number of
// violations; exit status 1 on any.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_2512_20269_gb300/csrc/dfloat.cuh"

using namespace iffd;

int main() {
  std::mt19937_64 g(1);
  std::uniform_real_distribution<double> u(-1, 1);
  std::uniform_int_distribution<int> ex(-74, 126);
  std::uniform_int_distribution<int> ex_small(-126, -75);
  double worst = 0;
  long bad = 0;
  for (long k = 0; k < 4000000; ++k) {
    double x = std::ldexp(u(g), ex(g));
    if (k % 97 == 0) x = 0.0;
    if (k % 101 == 0) x = -0.0;
    const df v = to_df(x);
    const double back = (double)v.hi + (double)v.lo;
    const double err = x == 0 ? std::fabs(back) : std::fabs(back - x) / std::fabs(x);
    if (err > worst) worst = err;
    if (err > std::ldexp(1.0, -47)) ++bad;
    if (x != 0 && v.hi != 0 && std::fabs(v.lo) > std::ldexp(1.0, std::ilogb(v.hi) - 23)) ++bad;
    if (std::signbit(x) != std::signbit(v.hi)) ++bad;
    if (to_double(v) != back) ++bad;
  }
  for (long k = 0; k < 200000; ++k) {
    // normal FP32 magnitudes in [2^-126, 2^-74)
    const double x = std::ldexp((u(g) < 0 ? -1.0 : 1.0) * (1.0 + 0.999 * std::fabs(u(g))), ex_small(g));
    const df v = to_df(x);
    const double back = (double)v.hi + (double)v.lo;
    if (x != 0 && std::fabs(back - x) > std::ldexp(std::fabs(x), -23)) ++bad;
  }
  std::uniform_int_distribution<unsigned> ub;
  for (long k = 0; k < 4000000; ++k) {
    const float f = float_of(ub(g));
    if (std::isnan(f)) continue;
    if (float_to_double_bits(f) != (double)f) ++bad;
  }
  std::printf("worst %.3e bad %ld\n", worst, bad);
  return bad != 0;
}
