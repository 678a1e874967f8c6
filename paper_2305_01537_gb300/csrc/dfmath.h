// tanh of an FP64 value in compensated FP32-pair arithmetic (about 48-bit significands), for the
// compensated-FP32 form's fused chain steps F(tanh z) and (1 - tanh^2 z) F^T g. The FP64 pipe of the
// target is about 60 times slower than FP32; a library tanh in FP64 costs more than the filter.
//
// Method (written from the definitions): with a = |x|,
//   a >= 19.1:  tanh a = 1 to FP64 rounding (1 - tanh a < 2^-54);
//   a >= 1/4:   e = exp(-2a) by base-2 range reduction, -2a log2(e) = n + f with n = rint and
//               |f| <= 1/2, exp(f ln 2) from its Taylor series to the term of degree 13, times 2^n;
//               tanh a = (1 - e) / (1 + e);
//   a < 1/4:    m = expm1(-2a) from its Taylor series to degree 16 (no cancellation);
//               tanh a = -m / (2 + m).
// Pair arithmetic uses Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based exact product; the
// division takes three quotient terms from the FP32 reciprocal, each remainder formed exactly. The
// input is split into a pair by integer bit operations (df32.h) and the result joined back the same
// way, so no FP64 instruction runs. Relative error below 2^-45 (host test against long double).
#pragma once

#include <cmath>
#include <cstdint>

#include "df32.h"

namespace sph {
namespace dfm {

// FP32 operations that the compiler must not contract into FMAs (the transformations rely on the
// rounding of each step).
DF_HD float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DF_HD float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DF_HD float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DF_HD float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

DF_HD df two_sum(float a, float b) {
  const float s = fadd(a, b);
  const float bb = fsub(s, a);
  return df{s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))};
}
DF_HD df fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = fadd(a, b);
  return df{s, fsub(b, fsub(s, a))};
}
DF_HD df add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(a.lo, b.lo)));
}
DF_HD df neg(df a) { return df{-a.hi, -a.lo}; }
DF_HD df mul(df a, df b) {
  const float p = fmul(a.hi, b.hi);
  float e = ffma(a.hi, b.hi, -p);
  e = ffma(a.hi, b.lo, e);
  e = ffma(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
DF_HD df mulf(df a, float b) {
  const float p = fmul(a.hi, b);
  return fast_two_sum(p, ffma(a.lo, b, ffma(a.hi, b, -p)));
}
DF_HD float frcp(float a) {  // correctly rounded 1 / a
#ifdef __CUDA_ARCH__
  return __frcp_rn(a);
#else
  return 1.0f / a;
#endif
}
// a / b (b.hi != 0): quotient terms q1 + q2 + q3 from y = 1 / b.hi, remainders exact.
DF_HD df div(df a, df b) {
  const float y = frcp(b.hi);
  const float q1 = fmul(a.hi, y);
  const df r1 = add(a, neg(mulf(b, q1)));
  const float q2 = fmul(r1.hi, y);
  const df r2 = add(r1, neg(mulf(b, q2)));
  const float q3 = fmul(r2.hi, y);
  const df q = fast_two_sum(q1, q2);
  return fast_two_sum(q.hi, fadd(q.lo, q3));
}
DF_HD df scale2(df a, int n) {  // a 2^n, n in [-100, 100], exact while the parts stay normal
  const float s = df_from_bits32((uint32_t)(n + 127) << 23);
  return df{fmul(a.hi, s), fmul(a.lo, s)};
}

// ln 2 and log2(e), and 1/k! (k = 0 .. 16), as pairs (high part the FP32 rounding, low part the
// FP32 rounding of the rest).
struct Consts {
  static constexpr float ln2_hi = 0x1.62e43p-1f, ln2_lo = -0x1.05c61p-29f;
  static constexpr float log2e_hi = 0x1.715476p+0f, log2e_lo = 0x1.4ae0cp-26f;
};
DF_HD df inv_fact(int k) {
  switch (k) {
    case 0: case 1: return df{1.0f, 0.0f};
    case 2: return df{0x1.0p-1f, 0.0f};
    case 3: return df{0x1.555556p-3f, -0x1.555556p-28f};
    case 4: return df{0x1.555556p-5f, -0x1.555556p-30f};
    case 5: return df{0x1.111112p-7f, -0x1.dddddep-32f};
    case 6: return df{0x1.6c16c2p-10f, -0x1.27d27ep-35f};
    case 7: return df{0x1.a01a02p-13f, -0x1.7f97fap-39f};
    case 8: return df{0x1.a01a02p-16f, -0x1.7f97fap-42f};
    case 9: return df{0x1.71de3ap-19f, 0x1.55b1ccp-45f};
    case 10: return df{0x1.27e4fcp-22f, -0x1.10ec14p-47f};
    case 11: return df{0x1.ae6456p-26f, 0x1.fd5138p-52f};
    case 12: return df{0x1.1eed8ep-29f, 0x1.ff1b12p-54f};
    case 13: return df{0x1.612462p-33f, -0x1.8af25ep-58f};
    case 14: return df{0x1.93974ap-37f, 0x1.180f94p-62f};
    case 15: return df{0x1.ae7f3ep-41f, 0x1.ccee08p-67f};
    default: return df{0x1.ae7f3ep-45f, 0x1.ccee08p-71f};
  }
}

// sum_{k=k0}^{K} u^k / k! / u^k0 by Horner's rule (u a pair).
template <int K, int K0>
DF_HD df taylor_tail(df u) {
  df p = inv_fact(K);
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int k = K - 1; k >= K0; --k) p = add(mul(p, u), inv_fact(k));
  return p;
}

}  // namespace dfm

// tanh(a) for a = |x| >= 2^-26 as a pair (the sign is applied by the callers).
DF_HD df df_tanh_abs(double x) {
  using namespace dfm;
  const uint64_t ab = df_bits64(x) & 0x7FFFFFFFFFFFFFFFull;
  if (ab >= 0x4033199999999999ull) return df{1.0f, 0.0f};  // a >= 19.1 (and infinities)
  const double a = df_from_bits64(ab);
  // a as a pair: a 2^-5 < 1 is split exactly by bit operations, then scaled back by 32
  const df A = scale2(df_from_double(a, 5), 5);
  if (ab < 0x3FD0000000000000ull) {  // a < 1/4: expm1(-2a) without cancellation
    const df u = df{-2.0f * A.hi, -2.0f * A.lo};
    const df m = mul(u, taylor_tail<16, 1>(u));  // u (1 + u/2! + ... ) = expm1(u)
    return div(neg(m), add(df{2.0f, 0.0f}, m));
  }
  // e = exp(-2a) = 2^n 2^f, -2a log2 e = n + f
  const df t = mul(df{-2.0f * A.hi, -2.0f * A.lo}, df{Consts::log2e_hi, Consts::log2e_lo});
#ifdef __CUDA_ARCH__
  const float nf = rintf(t.hi);
#else
  const float nf = std::nearbyint(t.hi);
#endif
  const df f = add(t, df{-nf, 0.0f});
  const df u = mul(f, df{Consts::ln2_hi, Consts::ln2_lo});
  const df e = scale2(add(df{1.0f, 0.0f}, mul(u, taylor_tail<13, 1>(u))), (int)nf);
  return div(add(df{1.0f, 0.0f}, neg(e)), add(df{1.0f, 0.0f}, e));
}

// |x| below 2^-26: tanh x = x and 1 - tanh^2 x = 1 to FP64 rounding (the next term is x^3/3).
DF_HD bool df_tanh_tiny(double x) { return (df_bits64(x) & 0x7FFFFFFFFFFFFFFFull) < 0x3E50000000000000ull; }

// tanh(x) to FP64 (NaN stays NaN).
DF_HD double df_tanh(double x) {
  const uint64_t b = df_bits64(x);
  if (((b >> 52) & 0x7ff) == 0x7ff && (b & 0xFFFFFFFFFFFFFull) != 0) return x;
  if (df_tanh_tiny(x)) return x;
  const double t = df_to_double(df_tanh_abs(x), 0);
  return (b >> 63) ? -t : t;
}

// 1 - tanh^2(x) = (1 - t)(1 + t) to FP64, t = tanh |x| (NaN stays NaN).
DF_HD double df_sech2(double x) {
  using namespace dfm;
  const uint64_t b = df_bits64(x);
  if (((b >> 52) & 0x7ff) == 0x7ff && (b & 0xFFFFFFFFFFFFFull) != 0) return x;
  if (df_tanh_tiny(x)) return 1.0;
  const df t = df_tanh_abs(x);
  return df_to_double(mul(add(df{1.0f, 0.0f}, neg(t)), add(df{1.0f, 0.0f}, t)), 0);
}

}  // namespace sph
