// Compensated FP32-pair ("double-float") numbers: a value is hi + lo with |lo| <= ulp(hi)/2, giving
// about 48 significant bits. Conversions to and from FP64 use integer bit operations only (no FP64
// instructions), with a per-block power-of-two scale 2^E chosen so that every scaled value is below
// 2 in magnitude. These helpers are __host__ __device__ so the host tests can check them bit for bit.
//
// Arithmetic follows the classical error-free transformations: Knuth's TwoSum, Dekker's
// FastTwoSum, and the FMA-based exact product (a*b = p + e with e = fma(a, b, -p)).
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace sph {

struct df {
  float hi, lo;
};

DF_HD uint64_t df_bits64(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}
DF_HD double df_from_bits64(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}
DF_HD uint32_t df_bits32(float x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
DF_HD float df_from_bits32(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
DF_HD float df_u2f(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(v);
#else
  return (float)v;
#endif
}

// Biased FP64 exponent field of x (0 for zero and subnormals).
DF_HD int df_exp_field(double x) { return (int)((df_bits64(x) >> 52) & 0x7ff); }

// x * 2^-E split into hi + lo. The top 24 significand bits go to hi, the next 29 (rounded to 24)
// to lo; values whose scaled exponent is below -100 (and FP64 subnormals) become 0, an error below
// 2^-100 of the block maximum. Requires x finite and |x| < 2^(E+1).
DF_HD df df_from_double(double x, int E) {
  const uint64_t u = df_bits64(x);
  const int bexp = (int)((u >> 52) & 0x7ff);
  const int es = bexp - 1023 - E;  // exponent of the scaled value
  df r{0.0f, 0.0f};
  if (bexp == 0 || es < -100) return r;
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const uint64_t mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const uint32_t mh = (uint32_t)(mant >> 29);  // 24 bits, leading bit set
  float hi = df_from_bits32(sign | ((uint32_t)(es + 127) << 23) | (mh & 0x7FFFFFu));
  const uint32_t rem = (uint32_t)(mant & 0x1FFFFFFFull);  // 29 bits below hi
  float lo = 0.0f;
  if (rem != 0 && es - 52 + 127 >= 1) {
    lo = df_u2f(rem) * df_from_bits32((uint32_t)(es - 52 + 127) << 23);
    if (sign) lo = -lo;
  }
  // renormalise so that |lo| <= ulp(hi)/2
  const float s = hi + lo;
  r.lo = lo - (s - hi);
  r.hi = s;
  return r;
}

// (hi + lo) * 2^E rounded toward zero to FP64 (error below 2^-52 relative). Zero and FP32
// subnormal parts are treated as zero. The result exponent must be in the FP64 normal range.
DF_HD double df_to_double(df v, int E) {
  const uint32_t hb = df_bits32(v.hi);
  const int eh = (int)((hb >> 23) & 0xff);
  if (eh == 0) return 0.0;
  uint64_t M = ((uint64_t)((hb & 0x7FFFFFu) | 0x800000u)) << 29;  // 53-bit frame, LSB = 2^(eh-179)
  const uint32_t lb = df_bits32(v.lo);
  const int el = (int)((lb >> 23) & 0xff);
  if (el != 0) {
    const uint64_t Ml = (uint64_t)((lb & 0x7FFFFFu) | 0x800000u);  // LSB = 2^(el-150)
    const int d = el - eh + 29;
    uint64_t A = 0;
    if (d >= 0) A = Ml << d;
    else if (d > -25) A = Ml >> (-d);
    if (((hb ^ lb) & 0x80000000u) == 0) M += A;
    else M -= A;
  }
  int e = eh - 127 + E;
  if (M >= (1ull << 53)) {
    M >>= 1;
    e += 1;
  } else if (M < (1ull << 52)) {
    M <<= 1;
    e -= 1;
  }
  if (e + 1023 <= 0) return 0.0;
  const uint64_t bits = ((uint64_t)(hb & 0x80000000u) << 32) | ((uint64_t)(e + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull);
  return df_from_bits64(bits);
}

}  // namespace sph
