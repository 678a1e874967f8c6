// Host check of the compensated FP32-pair tanh (dfmath.h) against long double tanhl: relative error
// of tanh and absolute error of 1 - tanh^2 over arguments from 1e-30 to 40, both signs, and the
// special values. Prints "ok <max rel err> <max abs err>" or the first failure.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>

#include "../paper_2305_01537_gb300/csrc/dfmath.h"

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> ue(-30.0, std::log10(40.0));
  double max_rel = 0.0, max_abs = 0.0, worst_x = 0.0;
  const double tol_rel = std::ldexp(1.0, -45), tol_abs = std::ldexp(1.0, -45);
  auto check = [&](double x) -> bool {
    const long double ref = tanhl((long double)x);
    const double got = sph::df_tanh(x);
    const long double den = fabsl(ref) > 0 ? fabsl(ref) : 1.0L;
    const double rel = (double)(fabsl((long double)got - ref) / den);
    const long double s2 = 1.0L - ref * ref;
    const double abs_err = (double)fabsl((long double)sph::df_sech2(x) - s2);
    if (rel > max_rel) {
      max_rel = rel;
      worst_x = x;
    }
    if (abs_err > max_abs) max_abs = abs_err;
    if (!(rel <= tol_rel) || !(abs_err <= tol_abs)) {
      std::printf("fail x=%.17g tanh=%.17g ref=%.17Lg rel=%.3g sech2 abs err=%.3g\n", x, got, ref, rel, abs_err);
      return false;
    }
    return true;
  };
  for (int i = 0; i < 2000000; ++i) {
    const double x = std::pow(10.0, ue(rng)) * ((i & 1) ? -1.0 : 1.0);
    if (!check(x)) return 1;
  }
  const double edges[] = {0.0, -0.0, 0.25, 0.2499999999999999, 0.2500000000000001, 19.1, 19.099999999999998,
                          1e-300, 5e-324, 0.5, 1.0, 2.0, 10.0, 18.0, 100.0, 1e300, INFINITY, -INFINITY};
  for (double x : edges)
    if (!check(x)) return 1;
  const double nan = std::nan("");
  if (!std::isnan(sph::df_tanh(nan)) || !std::isnan(sph::df_sech2(nan))) {
    std::printf("fail: NaN\n");
    return 1;
  }
  std::printf("ok %.3g %.3g worst at %.17g\n", max_rel, max_abs, worst_x);
  return 0;
}
