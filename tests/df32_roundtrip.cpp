// Host check of the FP64 <-> FP32-pair conversions of csrc/df32.h (compiled by test_df32_host.py).
// Prints one line per failure and "ok <count>" at the end.
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_2305_01537_gb300/csrc/df32.h"

using sph::df;

static int check(double x, int E, long& n) {
  ++n;
  const df v = sph::df_from_double(x, E);
  const long double scaled = std::ldexp((long double)x, -E);
  const long double got = (long double)v.hi + (long double)v.lo;
  // normalised pair
  if (v.hi != 0.0f && std::fabs((double)v.lo) > std::ldexp(std::fabs((double)v.hi), -24) * 1.0000001) {
    std::printf("not normalised x=%.17g E=%d hi=%.9g lo=%.9g\n", x, E, v.hi, v.lo);
    return 1;
  }
  const long double tol_in = std::fabs(scaled) * std::ldexp(1.0L, -47) + std::ldexp(1.0L, -100);
  if (std::fabs(got - scaled) > tol_in) {
    std::printf("from_double x=%.17g E=%d err=%Lg\n", x, E, std::fabs(got - scaled));
    return 1;
  }
  const double back = sph::df_to_double(v, E);
  const long double exact = std::ldexp(got, E);
  const long double tol_out = std::fabs(exact) * std::ldexp(1.0L, -52);
  if (std::fabs((long double)back - exact) > tol_out) {
    std::printf("to_double x=%.17g E=%d back=%.17g exact=%.21Lg\n", x, E, back, exact);
    return 1;
  }
  return 0;
}

int main() {
  std::mt19937_64 rng(2305);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-60, 60);
  long n = 0;
  int bad = 0;
  // random values with the block exponent E taken from the value itself or above it
  for (int t = 0; t < 200000 && bad < 20; ++t) {
    const double x = std::ldexp(u(rng), ex(rng));
    int e2;
    std::frexp(x, &e2);
    const int E = (e2 - 1) + (t % 7);  // |x| < 2^(E+1)
    bad += check(x, E, n);
  }
  // special values
  const double specials[] = {0.0, -0.0, 1.0, -1.0, 0.5, 1.9999999999999998, 3.0, 1e-300, -1e-300, 4.9e-324,
                             0.1, -0.7, 1.0 + std::ldexp(1.0, -52), 1.0 - std::ldexp(1.0, -53)};
  for (double x : specials) bad += check(x, 1, n);
  // exact pairs round-trip exactly when the value has at most 48 significant bits
  for (int t = 0; t < 10000; ++t) {
    const double x = std::ldexp(std::floor(u(rng) * std::ldexp(1.0, 47)), -47);
    const df v = sph::df_from_double(x, 0);
    if (sph::df_to_double(v, 0) != x) {
      std::printf("48-bit value not exact: %.17g\n", x);
      ++bad;
    }
    ++n;
  }
  if (bad) return 1;
  std::printf("ok %ld\n", n);
  return 0;
}
