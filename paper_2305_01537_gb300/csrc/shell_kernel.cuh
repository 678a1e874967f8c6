// Shell kernel of the double FFT filter (arXiv:2305.01537, Sec. II.C), staged (ping-pong) form.
// Included by shell_inst.cu, which the build compiles once per (precision, FFT length) pair.
//
// One CTA filters one (field, shell) pair; two CTAs share an SM where shared memory allows, so that
// one CTA's copies and barriers overlap the other's arithmetic. The shell (Ntheta x Nphi values) is
// staged once in shared memory: by bulk copies of its rows (TMA engine, one mbarrier) in the FP64
// form, by 16-byte cp.async in the compensated-FP32 form. The sequences of a pass are transformed
// in batches; the FFT stages ping-pong between the shell's own memory (each sequence's slots,
// below) and a scratch buffer with a linear layout: a thread reads a butterfly's inputs from one,
// writes its outputs to the other, and needs one barrier per stage.
//
//  theta pass (Sec. II.C, first filter equation, double covering): circle k (k < Nphi/2) is
//    c[q] = x[q][k] for q < Ntheta and (-1)^a x[2 Ntheta-1-q][k+Nphi/2] for q >= Ntheta. Circles
//    2s and 2s+1 form the real and imaginary parts of one complex sequence; their multipliers are
//    equal and real-even, so real and imaginary outputs are the two filtered circles. While the
//    sequence is being transformed, its 2 Ntheta complex slots are the value pairs
//    (x[j][2s], x[j][2s+1]) and (x[j][2s+h], x[j][2s+1+h]), h = Nphi/2.
//  phi pass (Sec. II.C, second filter equation): rings j and Ntheta-1-j (same m_max: sin is
//    symmetric about the equator) form one complex sequence; its Nphi complex slots are the value
//    pairs of the two rows. Rings whose multipliers differ (possible only for the sharp filter at
//    a cutoff boundary) take the exact two-real-FFT split W_m = (f1+f2)/2 Z_m + (f1-f2)/2 conj(Z_-m).
//  A lone circle (Nphi/2 odd) or lone middle ring (Ntheta odd) is transformed in an extra buffer.
//  Identity skipping: exponential and sharp filters keep every mode when l_max >= Ntheta (theta)
//    or m_max >= Nphi/2 (phi); those shells and rings are not transformed at all.
//  Hybrid fields (Sec. II.C, Jameson's shock detector): the detector runs on the FP64 shell before
//    anything else is decided; a circle or ring whose detector fired takes the Gaussian table, the
//    others the exponential one, and circle pairs or mirror rings that take different tables use
//    the exact two-real-FFT split above.
//
// Shared memory is addressed with 32-bit shared-window addresses. The first stage reads and the last
// stage writes the shell's own row-major layout (row stride Nphi + 2, so value pairs are 16-byte
// aligned); in between, a sequence's slots in the shell memory have their row (theta) or pair
// column (phi) index XOR-swizzled within groups of 8, and so does the scratch index, which keeps
// unit-stride and radix-stride accesses free of bank conflicts.
//
// The arithmetic policy is FP64 (F64) or compensated FP32 pairs (DF, about 48-bit significands,
// with a per-shell power-of-two scale). Multipliers f(|l|)/N and twiddles come from FP64 tables
// built on the host.
#pragma once

#include <type_traits>

#include "df32.h"
#include "dfmath.h"
#include "internal.h"

namespace sph {
namespace shellk {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ------------------------------------------------------------------ bulk copies (TMA engine)

constexpr long long kBarWaitLimit = 1LL << 24;  // bounded mbarrier polls (about a second at most)

__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One try of the phase with the given parity (acquire: the copies that completed it are visible).
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kBarWaitLimit; ++it)
    if (bar_try(bar, parity)) return true;
  return false;
}
// The phase's single arrival, with the bytes its copies will deliver.
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to this
// CTA's shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Thread 0 waits (bounded) for the shell's bulk copies; every thread then observes the completed
// phase. A wait that runs out latches SPH_ETIMEOUT and waits once more for the copies in flight;
// false (the same in every thread) if they never completed.
__device__ __forceinline__ bool wait_copies(unsigned* status, uint32_t bar, int* flag) {
  if (threadIdx.x == 0) {
    int bad = 0;
    if (!bar_wait(bar, 0)) {
      atomicCAS(status, 0u, (unsigned)SPH_ETIMEOUT);
      bad = bar_wait(bar, 0) ? 0 : 1;
    }
    *flag = bad;
  }
  __syncthreads();
  if (*flag) return false;
  bar_try(bar, 0);
  return true;
}

// ------------------------------------------------------------------ arithmetic policies

struct F64 {
  using T = double;
  struct C {
    double re, im;
  };
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T add_nr(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub_nr(T a, T b) { return a - b; }
  static __device__ __forceinline__ T norm(T a) { return a; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T half(T a) { return 0.5 * a; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T from_tab(const void* tab, size_t i) {
    return __ldg(static_cast<const double*>(tab) + i);
  }
  static __device__ __forceinline__ C cmul(C a, C w) {
    return C{fma(a.re, w.re, -a.im * w.im), fma(a.re, w.im, a.im * w.re)};
  }
  static __device__ __forceinline__ T ld8(uint32_t a) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
  }
  static __device__ __forceinline__ void st8(uint32_t a, T v) {
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
  }
  static __device__ __forceinline__ C ld16(uint32_t a) {
    double x, y;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a));
    return C{x, y};
  }
  static __device__ __forceinline__ void st16(uint32_t a, C v) {
    asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.re), "d"(v.im) : "memory");
  }
};

struct DF {
  using T = df;
  struct C {
    df re, im;
  };
  static __device__ __forceinline__ df add(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return df{h, __fsub_rn(e, __fsub_rn(h, s))};
  }
  static __device__ __forceinline__ df neg(df a) { return df{-a.hi, -a.lo}; }
  static __device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }
  // Sum without the final renormalisation: hi is the rounded sum of the high parts, lo collects
  // its exact rounding error and the low parts. Chains of these stay accurate to about 2^-46 as
  // long as each butterfly's outputs are renormalised (norm) before they are stored.
  static __device__ __forceinline__ df add_nr(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
  }
  static __device__ __forceinline__ df sub_nr(df a, df b) { return add_nr(a, neg(b)); }
  static __device__ __forceinline__ df norm(df a) {
    const float h = __fadd_rn(a.hi, a.lo);
    return df{h, __fsub_rn(a.lo, __fsub_rn(h, a.hi))};
  }
  // Product (exact high product plus the cross terms), not renormalised.
  static __device__ __forceinline__ df mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df{p, e};
  }
  static __device__ __forceinline__ df half(df a) { return df{0.5f * a.hi, 0.5f * a.lo}; }
  static __device__ __forceinline__ df zero() { return df{0.0f, 0.0f}; }
  static __device__ __forceinline__ df from_tab(const void* tab, size_t i) {
    const float2 v = __ldg(static_cast<const float2*>(tab) + i);
    return df{v.x, v.y};
  }
  // a*b - c*d in compensated arithmetic: exact products of the high parts, TwoSum of their
  // difference, the low-order cross terms accumulated by FMA (not renormalised).
  static __device__ __forceinline__ df dot2(df a, df b, df c, df d) {
    const float p1 = __fmul_rn(a.hi, b.hi);
    const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
    const float p2 = __fmul_rn(c.hi, d.hi);
    const float e2 = __fmaf_rn(c.hi, d.hi, -p2);
    const float s = __fsub_rn(p1, p2);
    const float bb = __fsub_rn(s, p1);
    const float err = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(-p2, bb));
    float t = __fadd_rn(__fsub_rn(e1, e2), err);
    t = __fmaf_rn(a.hi, b.lo, t);
    t = __fmaf_rn(a.lo, b.hi, t);
    t = __fmaf_rn(-c.hi, d.lo, t);
    t = __fmaf_rn(-c.lo, d.hi, t);
    return df{s, t};
  }
  static __device__ __forceinline__ C cmul(C a, C w) {
    return C{dot2(a.re, w.re, a.im, w.im), dot2(a.re, w.im, neg(a.im), w.re)};
  }
  static __device__ __forceinline__ T ld8(uint32_t a) {
    float x, y;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
    return df{x, y};
  }
  static __device__ __forceinline__ void st8(uint32_t a, T v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.hi), "f"(v.lo) : "memory");
  }
  static __device__ __forceinline__ C ld16(uint32_t a) {
    float x, y, z, w;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
    return C{df{x, y}, df{z, w}};
  }
  static __device__ __forceinline__ void st16(uint32_t a, C v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.re.hi), "f"(v.re.lo), "f"(v.im.hi),
                 "f"(v.im.lo)
                 : "memory");
  }
};

template <class P>
struct Cx {
  using C = typename P::C;
  using T = typename P::T;
  static __device__ __forceinline__ C add(C a, C b) { return C{P::add_nr(a.re, b.re), P::add_nr(a.im, b.im)}; }
  static __device__ __forceinline__ C sub(C a, C b) { return C{P::sub_nr(a.re, b.re), P::sub_nr(a.im, b.im)}; }
  static __device__ __forceinline__ C norm(C a) { return C{P::norm(a.re), P::norm(a.im)}; }
  static __device__ __forceinline__ C scale(C a, T g) { return C{P::mul(a.re, g), P::mul(a.im, g)}; }
  static __device__ __forceinline__ C neg(C a) { return C{P::neg(a.re), P::neg(a.im)}; }
  template <int DIR>  // multiply by DIR * i
  static __device__ __forceinline__ C mul_i(C v) {
    return DIR < 0 ? C{v.im, P::neg(v.re)} : C{P::neg(v.im), v.re};
  }
  static __device__ __forceinline__ C conj(C w) { return C{w.re, P::neg(w.im)}; }
  // -v if `flip`, else v. In FP64 the sign bits change by integer operations: a negation chosen
  // at run time would otherwise cost FP64 additions (the pipe that bounds the FP64 form).
  static __device__ __forceinline__ C neg_if(C v, bool flip) {
    if constexpr (std::is_same<T, double>::value) {
      const int m = (int)((unsigned)flip << 31);
      return C{__hiloint2double(__double2hiint(v.re) ^ m, __double2loint(v.re)),
               __hiloint2double(__double2hiint(v.im) ^ m, __double2loint(v.im))};
    } else {
      return flip ? neg(v) : v;
    }
  }
};

// Constants of the radix kernels in the policy's precision (from FP64 host values).
template <class P>
struct Consts {
  typename P::T c8;  // sqrt(1/2)
  typename P::T s3;  // sqrt(3)/2
};

// ------------------------------------------------------------------ in-register DFTs
// V[u] = sum_r v[r] exp(DIR 2 pi i u r / R), DIR = -1 forward, +1 inverse.

template <class P, int R, int DIR>
struct Dft;

template <class P, int DIR>
struct Dft<P, 2, DIR> {
  using X = Cx<P>;
  static __device__ __forceinline__ void run(typename P::C* v, const Consts<P>&) {
    const auto a = v[0], b = v[1];
    v[0] = X::add(a, b);
    v[1] = X::sub(a, b);
  }
};

template <class P, int DIR>
struct Dft<P, 4, DIR> {
  using X = Cx<P>;
  static __device__ __forceinline__ void run(typename P::C* v, const Consts<P>&) {
    const auto a = X::add(v[0], v[2]), b = X::sub(v[0], v[2]);
    const auto c = X::add(v[1], v[3]);
    const auto d = X::template mul_i<DIR>(X::sub(v[1], v[3]));
    v[0] = X::add(a, c);
    v[2] = X::sub(a, c);
    v[1] = X::add(b, d);
    v[3] = X::sub(b, d);
  }
};

template <class P, int DIR>
struct Dft<P, 8, DIR> {
  using X = Cx<P>;
  static __device__ __forceinline__ void run(typename P::C* v, const Consts<P>& k) {
    typename P::C e[4] = {v[0], v[2], v[4], v[6]};
    typename P::C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<P, 4, DIR>::run(e, k);
    Dft<P, 4, DIR>::run(o, k);
    // o[u] *= w8^u, w8 = exp(DIR i pi/4) = sqrt(1/2) (1 + DIR i)
    const typename P::C o1 = X::scale(X::add(o[1], X::template mul_i<DIR>(o[1])), k.c8);
    const typename P::C o2 = X::template mul_i<DIR>(o[2]);
    const typename P::C o3 = X::scale(X::sub(X::template mul_i<DIR>(o[3]), o[3]), k.c8);
    v[0] = X::add(e[0], o[0]);
    v[4] = X::sub(e[0], o[0]);
    v[1] = X::add(e[1], o1);
    v[5] = X::sub(e[1], o1);
    v[2] = X::add(e[2], o2);
    v[6] = X::sub(e[2], o2);
    v[3] = X::add(e[3], o3);
    v[7] = X::sub(e[3], o3);
  }
};

template <class P, int DIR>
struct Dft<P, 3, DIR> {
  using X = Cx<P>;
  static __device__ __forceinline__ void run(typename P::C* v, const Consts<P>& k) {
    const auto t = X::add(v[1], v[2]);
    const auto s = X::sub(v[1], v[2]);
    const typename P::C m{P::sub_nr(v[0].re, P::half(t.re)), P::sub_nr(v[0].im, P::half(t.im))};
    const auto w = X::template mul_i<DIR>(X::scale(s, k.s3));
    v[0] = X::add(v[0], t);
    v[1] = X::add(m, w);
    v[2] = X::sub(m, w);
  }
};

// FP64 radix-8 without twiddles: the two products by sqrt(1/2) fold into the output additions
// (one FMA per output component instead of a multiply and an addition). run_scaled multiplies the
// inputs by real factors mu_t first (the spectral multipliers of an inverse transform's first
// stage), folded into the first level: mu_t v_t +- mu_{t+4} v_{t+4} takes one multiply and two
// FMAs per component instead of two multiplies and two additions.
template <int DIR>
struct Dft<F64, 8, DIR> {
  using X = Cx<F64>;
  using C = F64::C;
  static __device__ __forceinline__ void run(C* v, const Consts<F64>& k) {
    C p[4], q[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      p[t] = X::add(v[t], v[t + 4]);
      q[t] = X::sub(v[t], v[t + 4]);
    }
    finish(v, p, q, k);
  }
  static __device__ __forceinline__ void run_scaled(C* v, const double* mu, const Consts<F64>& k) {
    C p[4], q[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double ar = mu[t] * v[t].re, ai = mu[t] * v[t].im;
      p[t] = C{fma(mu[t + 4], v[t + 4].re, ar), fma(mu[t + 4], v[t + 4].im, ai)};
      q[t] = C{fma(-mu[t + 4], v[t + 4].re, ar), fma(-mu[t + 4], v[t + 4].im, ai)};
    }
    finish(v, p, q, k);
  }
  // the rest from the first level p_t = v_t + v_{t+4}, q_t = v_t - v_{t+4}: the 4-point transforms
  // of the even inputs (p0, q0, p2, q2) and of the odd ones (p1, q1, p3, q3), then the radix-2
  // combination with the eighth roots
  static __device__ __forceinline__ void finish(C* v, const C* p, const C* q, const Consts<F64>& k) {
    const C de = X::template mul_i<DIR>(q[2]), dd = X::template mul_i<DIR>(q[3]);
    const C e0 = X::add(p[0], p[2]), e2 = X::sub(p[0], p[2]), e1 = X::add(q[0], de), e3 = X::sub(q[0], de);
    const C o0 = X::add(p[1], p[3]), o2 = X::sub(p[1], p[3]), o1 = X::add(q[1], dd), o3 = X::sub(q[1], dd);
    // w8 o1 = sqrt(1/2) (o1 + DIR i o1), w8^2 o2 = DIR i o2, w8^3 o3 = sqrt(1/2) (DIR i o3 - o3)
    const C g1 = X::add(o1, X::template mul_i<DIR>(o1));
    const C r2 = X::template mul_i<DIR>(o2);
    const C g3 = X::sub(X::template mul_i<DIR>(o3), o3);
    const double c = k.c8;
    v[0] = X::add(e0, o0);
    v[4] = X::sub(e0, o0);
    v[1] = C{fma(c, g1.re, e1.re), fma(c, g1.im, e1.im)};
    v[5] = C{fma(-c, g1.re, e1.re), fma(-c, g1.im, e1.im)};
    v[2] = X::add(e2, r2);
    v[6] = X::sub(e2, r2);
    v[3] = C{fma(c, g3.re, e3.re), fma(c, g3.im, e3.im)};
    v[7] = C{fma(-c, g3.re, e3.re), fma(-c, g3.im, e3.im)};
  }
};

// ------------------------------------------------------------------ FP64 twiddled butterflies
// A twiddled radix-R stage (R = 2, 4, 8) in FP64 runs as log2 R levels of radix-2 butterflies
// a +- z b, each z a power of the stage twiddle w = exp(-2 pi i kk / (Ns R)) (conjugated for the
// inverse) times a power of i, which costs nothing. Every z is stored as a pair (m, r):
//   tangent form (|Re z| >= |Im z|):   z = m (1 + i r),    m = Re z, r = Im z / Re z;
//   cotangent form (|Im z| > |Re z|):  z = i m (1 + i r),  m = Im z, r = -Re z / Im z;
// so that with g = b + i r b (two FMAs) z b = m g or i m g, and both outputs a +- z b take one
// FMA per component: six FP64 operations per butterfly instead of ten (complex product and two
// complex additions). |r| <= 1 in both forms, so g carries no cancellation. The lowest significand
// bit of m marks the cotangent form (a change of at most one unit in the last place of m).
//
// The factorisation: with x_t = w^t v_t and omega = exp(DIR 2 pi i / 8),
//   V_u = sum_t x_t omega^(t u) = sum_{t<4} w^t omega^(t u) (v_t + (-1)^u w^4 v_{t+4}),
// so the first level pairs v_t with v_{t+4} under z = w^4; the even outputs are then a twiddled
// 4-point transform with twiddle w, the odd outputs one with twiddle w omega. A twiddled 4-point
// transform with twiddle y pairs q_a with q_{a+2} under y^2, then combines r_0 with r_1 under y
// (outputs 0 and 2) and under y DIR i (outputs 1 and 3). The table holds, per kk, w^4, w^2, w and
// w omega for R = 8; w^2 and w for R = 4; w for R = 2 (in the stage's R - 1 slots).
// The conjugate (inverse) has r of the other sign, and in the cotangent form m of the other sign
// too; the sign of r goes into the FMAs' operand modifiers. With mx the factor of the real output
// component (z b = (mx x, m y) below): forward, m as stored and mx = -m in the cotangent form;
// inverse, mx = m as stored and m = -m in the cotangent form. Those sign changes flip the sign bit
// with an integer operation (a negation of a selected FP64 value would cost an FP64 addition).
struct Tw {
  double m, mx, r;
  bool cot;
};

template <int DIR>
__device__ __forceinline__ Tw tw_load(uint32_t a) {
  const F64::C e = F64::ld16(a);
  const int lo = __double2loint(e.re), hi = __double2hiint(e.re);
  const double flipped = __hiloint2double(hi ^ (int)((unsigned)(lo & 1) << 31), lo);  // -m if cotangent
  if (DIR < 0) return Tw{e.re, flipped, e.im, (lo & 1) != 0};
  return Tw{flipped, e.re, e.im, (lo & 1) != 0};
}

// (a, b) <- (a + z b, a - z b)
template <int DIR>
__device__ __forceinline__ void tw_bfly(F64::C& a, F64::C& b, const Tw& z) {
  // g = b + i r b (r of the conjugate's sign for the inverse)
  const double gre = DIR < 0 ? fma(-z.r, b.im, b.re) : fma(z.r, b.im, b.re);
  const double gim = DIR < 0 ? fma(z.r, b.re, b.im) : fma(-z.r, b.re, b.im);
  const double x = z.cot ? gim : gre;
  const double y = z.cot ? gre : gim;
  const F64::C a0 = a;
  a = F64::C{fma(z.mx, x, a0.re), fma(z.m, y, a0.im)};
  b = F64::C{fma(-z.mx, x, a0.re), fma(-z.m, y, a0.im)};
}

template <int R, int DIR>
struct TwDft;

template <int DIR>
struct TwDft<2, DIR> {
  static __device__ __forceinline__ void run(F64::C* v, uint32_t tw) { tw_bfly<DIR>(v[0], v[1], tw_load<DIR>(tw)); }
};

template <int DIR>
struct TwDft<4, DIR> {
  using X = Cx<F64>;
  static __device__ __forceinline__ void run(F64::C* v, uint32_t tw) {
    const Tw z2 = tw_load<DIR>(tw), z1 = tw_load<DIR>(tw + 16u);
    tw_bfly<DIR>(v[0], v[2], z2);
    tw_bfly<DIR>(v[1], v[3], z2);
    F64::C b = X::template mul_i<DIR>(v[3]);
    tw_bfly<DIR>(v[0], v[1], z1);  // outputs 0, 2
    tw_bfly<DIR>(v[2], b, z1);     // outputs 1, 3
    const F64::C u2 = v[1];
    v[1] = v[2];
    v[2] = u2;
    v[3] = b;
  }
};

template <int DIR>
struct TwDft<8, DIR> {
  using X = Cx<F64>;
  static __device__ __forceinline__ void run(F64::C* v, uint32_t tw) {
    const Tw z4 = tw_load<DIR>(tw), z2 = tw_load<DIR>(tw + 16u);
    const Tw z1 = tw_load<DIR>(tw + 32u), z1w = tw_load<DIR>(tw + 48u);
#pragma unroll
    for (int t = 0; t < 4; ++t) tw_bfly<DIR>(v[t], v[t + 4], z4);
    // even outputs: twiddled 4-point transform of v[0..3] with twiddle w
    tw_bfly<DIR>(v[0], v[2], z2);
    tw_bfly<DIR>(v[1], v[3], z2);
    F64::C be = X::template mul_i<DIR>(v[3]);
    tw_bfly<DIR>(v[0], v[1], z1);  // V0, V4
    tw_bfly<DIR>(v[2], be, z1);    // V2, V6
    // odd outputs: twiddled 4-point transform of v[4..7] with twiddle w omega ((w omega)^2 = w^2 DIR i)
    F64::C b6 = X::template mul_i<DIR>(v[6]);
    F64::C b7 = X::template mul_i<DIR>(v[7]);
    tw_bfly<DIR>(v[4], b6, z2);
    tw_bfly<DIR>(v[5], b7, z2);
    F64::C bo = X::template mul_i<DIR>(b7);
    tw_bfly<DIR>(v[4], v[5], z1w);  // V1, V5
    tw_bfly<DIR>(b6, bo, z1w);      // V3, V7
    const F64::C V1 = v[4], V2 = v[2], V4 = v[1], V5 = v[5];
    v[1] = V1;
    v[2] = V2;
    v[3] = b6;
    v[4] = V4;
    v[5] = V5;
    v[6] = be;
    v[7] = bo;
  }
};

// Stages whose twiddles use the FMA form: FP64 with radix 2, 4 or 8.
template <class P, int R>
__host__ __device__ constexpr bool fma_twiddles() {
  return std::is_same<P, F64>::value && (R == 2 || R == 4 || R == 8);
}

// The chain steps' pointwise maps, tanh and its derivative 1 - tanh^2, in the form's arithmetic:
// FP64 for the FP64 form, compensated FP32 pairs (dfmath.h) for the compensated-FP32 form.
template <class P>
__device__ __forceinline__ double map_tanh(double x) {
  if constexpr (std::is_same<P, DF>::value) return df_tanh(x);
  else return tanh(x);
}
template <class P>
__device__ __forceinline__ double map_sech2(double x) {
  if constexpr (std::is_same<P, DF>::value) {
    return df_sech2(x);
  } else {
    const double t = tanh(x);
    return 1.0 - t * t;
  }
}

// ------------------------------------------------------------------ pass accessors

// XOR swizzle of an index within aligned groups of 8 (identity past the last full group).
__device__ __forceinline__ int swz(int r, int full8) { return r < full8 ? (r ^ ((r >> 3) & 7)) : r; }

template <class P>
struct ThetaAcc {
  using C = typename P::C;
  using T = typename P::T;
  struct Seq {
    int b;
    bool lone;
    bool general;  // hybrid field: the two circles take different tables (exact split)
    bool alt;      // hybrid field: both circles take the second (Gaussian) table
  };
  uint32_t S;    // shell, row stride ld (8-byte elements)
  uint32_t ov;   // lone-circle slots (16-byte complex)
  uint32_t lin;  // scratch: sequence b, index n at (b - b0) * M + swizzled n
  uint32_t g;    // multipliers f(|l|)/M, l = 0..Ntheta; a hybrid field's Gaussian row follows
  const unsigned char* sel;   // hybrid field, per sequence: 0 first table, 1 second, 2 mixed
  const unsigned char* circ;  // hybrid field, per circle: 1 = second table
  bool hyb;
  int ld, Nth, Nth8, h, M, M8, nseq, b0;
  bool lone_last;  // Nphi/2 odd: the last sequence holds circle h-1 alone
  bool odd;        // parity a = 1
  bool hodd;       // h odd: pairs at column 2s+h are only 8-byte aligned

  __device__ __forceinline__ uint32_t el(int row, int col) const { return S + (uint32_t)(row * ld + col) * 8u; }
  __device__ __forceinline__ Seq seq(int b) const {
    const bool lone = lone_last && b == nseq - 1;
    if (!hyb) return Seq{b, lone, false, false};
    const int t = sel[b];
    return Seq{b, lone, t == 2, t == 1};
  }
  __device__ __forceinline__ int seq_len() const { return M; }
  __device__ __forceinline__ C pair_ld(uint32_t a, bool split) const {
    return split ? C{P::ld8(a), P::ld8(a + 8)} : P::ld16(a);
  }
  __device__ __forceinline__ void pair_st(uint32_t a, bool split, C v) const {
    if (split) {
      P::st8(a, v.re);
      P::st8(a + 8, v.im);
    } else {
      P::st16(a, v);
    }
  }
  // intermediate slot n of a sequence: swizzled row, the sequence's column pair
  __device__ __forceinline__ C slot_ld(const Seq& s, int n) const {
    if (s.lone) return P::ld16(ov + 16u * n);
    const bool up = n < Nth;
    const int r = up ? n : n - Nth;
    return pair_ld(el(swz(r, Nth8), up ? 2 * s.b : 2 * s.b + h), hodd && !up);
  }
  __device__ __forceinline__ void slot_st(const Seq& s, int n, C v) const {
    if (s.lone) {
      P::st16(ov + 16u * n, v);
      return;
    }
    const bool up = n < Nth;
    const int r = up ? n : n - Nth;
    pair_st(el(swz(r, Nth8), up ? 2 * s.b : 2 * s.b + h), hodd && !up, v);
  }
  // circle sample q, read from the shell's own layout with the parity sign past the pole
  __device__ __forceinline__ C gather(const Seq& s, int q) const {
    const bool up = q < Nth;
    const uint32_t a = el(up ? q : M - 1 - q, up ? 2 * s.b : 2 * s.b + h);
    const C v = s.lone ? C{P::ld8(a), P::zero()} : pair_ld(a, hodd && !up);
    return Cx<P>::neg_if(v, !up && odd);
  }
  __device__ __forceinline__ void scatter(const Seq& s, int q, C v) const {
    const bool up = q < Nth;
    v = Cx<P>::neg_if(v, !up && odd);
    const uint32_t a = el(up ? q : M - 1 - q, up ? 2 * s.b : 2 * s.b + h);
    if (s.lone) P::st8(a, v.re);
    else pair_st(a, hodd && !up, v);
  }
  __device__ __forceinline__ T mult(const Seq& s, int l) const {
    return P::ld8(g + (s.alt ? 8u * (uint32_t)(Nth + 1) : 0u) + 8u * (l <= Nth ? l : M - l));
  }
  // multipliers of the sequence's circles 2b and 2b+1 (split multiply of a mixed pair)
  __device__ __forceinline__ void mult2(const Seq& s, int l, T& f1, T& f2) const {
    const uint32_t alt = 8u * (uint32_t)(Nth + 1), o = 8u * (uint32_t)(l <= Nth ? l : M - l);
    f1 = P::ld8(g + (circ[2 * s.b] ? alt : 0u) + o);
    f2 = P::ld8(g + (circ[2 * s.b + 1] ? alt : 0u) + o);
  }
  __device__ __forceinline__ uint32_t lin_at(int b, int n) const {
    return lin + 16u * (uint32_t)((b - b0) * M + swz(n, M8));
  }
  __device__ __forceinline__ C lin_ld(int b, int n) const { return P::ld16(lin_at(b, n)); }
  __device__ __forceinline__ void lin_st(int b, int n, C v) const { P::st16(lin_at(b, n), v); }
  // sizes known at compile time for the fixed lengths (2 Ntheta = Nphi = LEN); SPLIT: the CTA
  // holds half of the meridians (a cluster pair shares the shell), i.e. a shell of Nphi/2 columns
  template <int LEN, bool SPLIT = false>
  __device__ __forceinline__ void fix() {
    if constexpr (LEN > 0) {
      constexpr int W = SPLIT ? LEN / 2 : LEN;  // columns held
      Nth = LEN / 2;
      Nth8 = (LEN / 2) & ~7;
      ld = W + 2;
      h = W / 2;
      M = LEN;
      M8 = LEN & ~7;
      nseq = (W / 2 + 1) / 2;
      lone_last = hodd = ((W / 2) & 1) != 0;
    }
  }
};

template <class P>
struct PhiAcc {
  using C = typename P::C;
  using T = typename P::T;
  struct Seq {
    int j1, j2;  // j2 < 0: lone middle ring
    bool general;
    bool alt1, alt2;  // hybrid field: ring j1 / j2 takes the second (Gaussian) table
  };
  uint32_t S, ov;
  uint32_t lin;       // scratch: sequence b, index n at (b - b0) * N + swizzled n
  const int2* pairs;  // (j1 | general << 30 | alt1 << 29 | alt2 << 28, j2) in shared memory
  const void* gtab;   // multipliers f(|m|)/Nphi of this shell: [Ntheta][Nphi/2+1] (global)
  size_t gbase, gbase_alt;  // the shell's rows of the first and the second table
  bool hyb;                 // hybrid field: the alt bits select the table
  int ld, N, N8, hN, hN8, nh, b0;

  __device__ __forceinline__ uint32_t el(int row, int col) const { return S + (uint32_t)(row * ld + col) * 8u; }
  __device__ __forceinline__ Seq seq(int b) const {
    const int2 p = pairs[b];
    return Seq{p.x & 0x0fffffff, p.y, ((p.x >> 30) & 1) != 0, hyb && ((p.x >> 29) & 1) != 0,
               hyb && ((p.x >> 28) & 1) != 0};
  }
  __device__ __forceinline__ int seq_len() const { return N; }
  __device__ __forceinline__ uint32_t slot(const Seq& s, int n) const {
    const bool lo = n < hN;
    const int u = lo ? n : n - hN;
    return el(lo ? s.j1 : s.j2, 2 * swz(u, hN8));
  }
  __device__ __forceinline__ C slot_ld(const Seq& s, int n) const {
    return s.j2 < 0 ? P::ld16(ov + 16u * n) : P::ld16(slot(s, n));
  }
  __device__ __forceinline__ void slot_st(const Seq& s, int n, C v) const {
    if (s.j2 < 0) P::st16(ov + 16u * n, v);
    else P::st16(slot(s, n), v);
  }
  __device__ __forceinline__ C gather(const Seq& s, int k) const {
    return C{P::ld8(el(s.j1, k)), s.j2 >= 0 ? P::ld8(el(s.j2, k)) : P::zero()};
  }
  __device__ __forceinline__ void scatter(const Seq& s, int k, C v) const {
    P::st8(el(s.j1, k), v.re);
    if (s.j2 >= 0) P::st8(el(s.j2, k), v.im);
  }
  __device__ __forceinline__ T ring_mult(int j, int m, bool alt) const {
    return P::from_tab(gtab, (alt ? gbase_alt : gbase) + (size_t)j * nh + (m <= hN ? m : N - m));
  }
  __device__ __forceinline__ T mult(const Seq& s, int m) const { return ring_mult(s.j1, m, s.alt1); }
  __device__ __forceinline__ void mult2(const Seq& s, int m, T& f1, T& f2) const {
    f1 = ring_mult(s.j1, m, s.alt1);
    f2 = ring_mult(s.j2, m, s.alt2);
  }
  __device__ __forceinline__ uint32_t lin_at(int b, int n) const {
    return lin + 16u * (uint32_t)((b - b0) * N + swz(n, N8));
  }
  __device__ __forceinline__ C lin_ld(int b, int n) const { return P::ld16(lin_at(b, n)); }
  __device__ __forceinline__ void lin_st(int b, int n, C v) const { P::st16(lin_at(b, n), v); }
  template <int LEN>
  __device__ __forceinline__ void fix() {
    if constexpr (LEN > 0) {
      ld = LEN + 2;
      N = LEN;
      N8 = LEN & ~7;
      hN = LEN / 2;
      hN8 = (LEN / 2) & ~7;
      nh = LEN / 2 + 1;
    }
  }
};

// Phi pass of a CTA that shares its shell with a cluster peer. The CTA of rank r owns the ring
// pairs (j, Ntheta-1-j) with j in [r Ntheta/4, (r+1) Ntheta/4). Its buffer A holds every row for
// the meridian blocks {r, r+2} (blocks of Nphi/4 columns), buffer B holds its own rows for the
// peer's blocks {1-r, 3-r}; inside each, a block pair sits at local columns [0, Nphi/2).
template <class P>
struct PhiSplitAcc {
  using C = typename P::C;
  using T = typename P::T;
  using Seq = typename PhiAcc<P>::Seq;
  uint32_t A, Bm;
  uint32_t lin0, lin1;  // scratch: the peer's rows of A (two blocks of `cap` sequences each)
  int cap;
  const int2* pairs;
  const void* gtab;
  size_t gbase, gbase_alt;  // the shell's rows of the first and the second table
  bool hyb;                 // hybrid field: the alt bits select the table
  int ld, N, N8, QB, QB8, Nth, r, hN, nh, b0;

  __device__ __forceinline__ int brow(int j) const {
    const int q = Nth / 4;
    return j < Nth / 2 ? j - q * r : q + (j - (Nth - (r + 1) * q));
  }
  __device__ __forceinline__ uint32_t el(int j, int c) const {
    const int blk = c / QB;
    const int lc = (c - blk * QB) + (blk >= 2 ? QB : 0);
    const bool mine = blk == r || blk == 2 + r;
    return mine ? A + (uint32_t)(j * ld + lc) * 8u : Bm + (uint32_t)(brow(j) * ld + lc) * 8u;
  }
  __device__ __forceinline__ Seq seq(int b) const {
    const int2 p = pairs[b];
    return Seq{p.x & 0x0fffffff, p.y, ((p.x >> 30) & 1) != 0, hyb && ((p.x >> 29) & 1) != 0,
               hyb && ((p.x >> 28) & 1) != 0};
  }
  __device__ __forceinline__ int seq_len() const { return N; }
  // slots: segments of Nphi/4 complex in A row j1, B row j1, A row j2, B row j2
  __device__ __forceinline__ uint32_t slot(const Seq& s, int n) const {
    const int seg = n / QB, u = n - seg * QB;
    const int j = seg < 2 ? s.j1 : s.j2;
    const int col = 2 * swz(u, QB8);
    return (seg & 1) ? Bm + (uint32_t)(brow(j) * ld + col) * 8u : A + (uint32_t)(j * ld + col) * 8u;
  }
  __device__ __forceinline__ C slot_ld(const Seq& s, int n) const { return P::ld16(slot(s, n)); }
  __device__ __forceinline__ void slot_st(const Seq& s, int n, C v) const { P::st16(slot(s, n), v); }
  __device__ __forceinline__ C gather(const Seq& s, int k) const {
    return C{P::ld8(el(s.j1, k)), P::ld8(el(s.j2, k))};
  }
  __device__ __forceinline__ void scatter(const Seq& s, int k, C v) const {
    P::st8(el(s.j1, k), v.re);
    P::st8(el(s.j2, k), v.im);
  }
  __device__ __forceinline__ T ring_mult(int j, int m, bool alt) const {
    return P::from_tab(gtab, (alt ? gbase_alt : gbase) + (size_t)j * nh + (m <= hN ? m : N - m));
  }
  __device__ __forceinline__ T mult(const Seq& s, int m) const { return ring_mult(s.j1, m, s.alt1); }
  __device__ __forceinline__ void mult2(const Seq& s, int m, T& f1, T& f2) const {
    f1 = ring_mult(s.j1, m, s.alt1);
    f2 = ring_mult(s.j2, m, s.alt2);
  }
  __device__ __forceinline__ uint32_t lin_at(int b, int n) const {
    const int bl = b - b0;
    const bool second = bl >= cap;
    return (second ? lin1 : lin0) + 16u * (uint32_t)((second ? bl - cap : bl) * N + swz(n, N8));
  }
  __device__ __forceinline__ C lin_ld(int b, int n) const { return P::ld16(lin_at(b, n)); }
  __device__ __forceinline__ void lin_st(int b, int n, C v) const { P::st16(lin_at(b, n), v); }
  template <int LEN>
  __device__ __forceinline__ void fix() {
    if constexpr (LEN > 0) {
      ld = LEN / 2 + 2;
      N = LEN;
      N8 = LEN & ~7;
      QB = LEN / 4;
      QB8 = (LEN / 4) & ~7;
      Nth = LEN / 2;
      hN = LEN / 2;
      nh = LEN / 2 + 1;
    }
  }
};

// ------------------------------------------------------------------ FFT stage

enum { kFirst = 1, kLast = 2, kMul = 4 };

// One radix-R Stockham stage over all B sequences: from the shell slots to the scratch (FROM_SLOTS)
// or back. tw is the stage's own twiddle table of Ns (R - 1) entries, R - 1 per kk: entry
// kk (R - 1) + t - 1 holds exp(-2 pi i t kk / (Ns R)) (compensated FP32 and radix 3), or the FP64
// FMA-form factors of TwDft in the first slots of kk's group (FP64, R = 2, 4, 8). A butterfly's
// twiddles are adjacent and the threads of a quarter warp (kk consecutive) read entries R - 1
// apart: different banks for R = 2, 4, 8. kFirst reads the logical sequence out of the shell
// layout, kLast writes it back there, kMul multiplies each input by the spectral multiplier
// (sequences flagged `general` were multiplied before, by general_multiply).
template <class P, class Acc, int R, int DIR, int MODE, bool FROM_SLOTS>
__device__ __forceinline__ void stage(const Acc& A, int N, int B, int Ns, uint32_t tw, const Consts<P>& k) {
  using C = typename P::C;
  using X = Cx<P>;
  const int NR = N / R;
  const int total = B * NR;
#pragma unroll 1
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int bl = w / NR, j = w - bl * NR;
    const int b = A.b0 + bl;
    const int kk = j % Ns;
    const auto sq = A.seq(b);
    // FP64 radix 8: the multipliers fold into the transform's first level (run_scaled)
    constexpr bool fold_mul = (MODE & kMul) && std::is_same<P, F64>::value && R == 8;
    C v[R];
    double mu[fold_mul ? R : 1];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int n = j + t * NR;
      C x = (MODE & kFirst) ? A.gather(sq, n) : (FROM_SLOTS ? A.slot_ld(sq, n) : A.lin_ld(b, n));
      if constexpr (fold_mul) mu[t] = sq.general ? 1.0 : A.mult(sq, n);
      else if ((MODE & kMul) && !sq.general) x = X::scale(x, A.mult(sq, n));
      v[t] = x;
    }
    if constexpr (fold_mul) {
      // kMul marks an inverse transform's first stage, which has no twiddles (Ns = 1)
      Dft<F64, 8, DIR>::run_scaled(v, mu, k);
    } else if constexpr (fma_twiddles<P, R>()) {
      if (Ns > 1) TwDft<R, DIR>::run(v, tw + 16u * (uint32_t)(kk * (R - 1)));
      else Dft<P, R, DIR>::run(v, k);
    } else {
      if (Ns > 1) {
#pragma unroll
        for (int t = 1; t < R; ++t) {
          C wt = P::ld16(tw + 16u * (uint32_t)(kk * (R - 1) + t - 1));
          if (DIR > 0) wt = X::conj(wt);
          v[t] = P::cmul(v[t], wt);
        }
      }
      Dft<P, R, DIR>::run(v, k);
    }
    const int base = (j / Ns) * Ns * R + kk;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int n = base + t * Ns;
      v[t] = X::norm(v[t]);
      if (MODE & kLast) A.scatter(sq, n, v[t]);
      else if (FROM_SLOTS) A.lin_st(b, n, v[t]);
      else A.slot_st(sq, n, v[t]);
    }
  }
  __syncthreads();
}

// Generic lengths: each stage is its own function, so one radix's register allocation does not
// weigh on the others (the call costs a register save and restore per stage).
template <class P, class Acc, int R, int DIR, int MODE>
__device__ __noinline__ void stage_ni(const Acc A, int N, int B, int Ns, uint32_t tw, const Consts<P> k,
                                      bool from_slots) {
  if (from_slots) stage<P, Acc, R, DIR, MODE, true>(A, N, B, Ns, tw, k);
  else stage<P, Acc, R, DIR, MODE, false>(A, N, B, Ns, tw, k);
}

template <class P, class Acc, int DIR, int MODE>
__device__ __forceinline__ void stage_r(int R, const Acc& A, int N, int B, int Ns, uint32_t tw, const Consts<P>& k,
                                        bool from_slots) {
  switch (R) {
    case 8: stage_ni<P, Acc, 8, DIR, MODE>(A, N, B, Ns, tw, k, from_slots); break;
    case 4: stage_ni<P, Acc, 4, DIR, MODE>(A, N, B, Ns, tw, k, from_slots); break;
    case 2: stage_ni<P, Acc, 2, DIR, MODE>(A, N, B, Ns, tw, k, from_slots); break;
    default: stage_ni<P, Acc, 3, DIR, MODE>(A, N, B, Ns, tw, k, from_slots); break;
  }
}

// Exact two-real-sequence multiply for sequences whose two halves take different multipliers:
// W_m = (f1+f2)/2 Z_m + (f1-f2)/2 conj(Z_{N-m}), on the spectrum held in the slots or the scratch.
// Used for mirror rings whose cutoffs differ beyond rounding and, for hybrid fields, for circle
// pairs and mirror rings of which one takes the Gaussian filter and the other the exponential.
template <class P, class Acc>
__device__ void general_multiply(const Acc& A, int B, bool in_slots) {
  using C = typename P::C;
  const int N = A.seq_len();
  const int nh = N / 2 + 1;
  for (int base = 0; base < B * nh; base += blockDim.x) {
    const int w = base + threadIdx.x;
    bool act = false;
    int m = 0, mn = 0, bb = 0;
    typename Acc::Seq sq{};
    C wm, wn;
    if (w < B * nh) {
      bb = A.b0 + w / nh;
      m = w - (w / nh) * nh;
      sq = A.seq(bb);
      act = sq.general;
      if (act) {
        mn = (N - m) % N;
        const C zm = in_slots ? A.slot_ld(sq, m) : A.lin_ld(bb, m);
        const C zn = in_slots ? A.slot_ld(sq, mn) : A.lin_ld(bb, mn);
        typename P::T f1, f2;
        A.mult2(sq, m, f1, f2);
        const auto ca = P::half(P::add(f1, f2)), cd = P::half(P::sub(f1, f2));
        wm = C{P::add(P::mul(zm.re, ca), P::mul(zn.re, cd)), P::sub(P::mul(zm.im, ca), P::mul(zn.im, cd))};
        wn = C{P::add(P::mul(zn.re, ca), P::mul(zm.re, cd)), P::sub(P::mul(zn.im, ca), P::mul(zm.im, cd))};
      }
    }
    __syncthreads();
    if (act) {
      if (in_slots) {
        A.slot_st(sq, m, wm);
        if (mn != m) A.slot_st(sq, mn, wn);
      } else {
        A.lin_st(bb, m, wm);
        if (mn != m) A.lin_st(bb, mn, wn);
      }
    }
    __syncthreads();
  }
}

// Runtime radix sequence (generic lengths).
template <class P, class Acc>
__device__ void pass_rt(const Acc& A, int N, int B, const Factors& f, uint32_t tw, const Consts<P>& k,
                        bool has_general) {
  // stage g (0-based over forward and inverse) reads the slots when g is even
  int Ns = 1;
  uint32_t ts = tw;  // the stage's twiddle table (Ns (R - 1) entries)
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    if (s == 0) stage_r<P, Acc, -1, kFirst>(R, A, N, B, Ns, ts, k, true);
    else stage_r<P, Acc, -1, 0>(R, A, N, B, Ns, ts, k, (s & 1) == 0);
    ts += 16u * (uint32_t)(Ns * (R - 1));
    Ns *= R;
  }
  if (has_general) general_multiply<P, Acc>(A, B, (f.nst & 1) == 0);
  Ns = 1;
  ts = tw;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    const bool first = s == 0, last = s == f.nst - 1;
    const bool from_slots = ((f.nst + s) & 1) == 0;
    if (first && last) stage_r<P, Acc, 1, kMul | kLast>(R, A, N, B, Ns, ts, k, from_slots);
    else if (first) stage_r<P, Acc, 1, kMul>(R, A, N, B, Ns, ts, k, from_slots);
    else if (last) stage_r<P, Acc, 1, kLast>(R, A, N, B, Ns, ts, k, from_slots);
    else stage_r<P, Acc, 1, 0>(R, A, N, B, Ns, ts, k, from_slots);
    ts += 16u * (uint32_t)(Ns * (R - 1));
    Ns *= R;
  }
}

// Compile-time radix sequence (fixed lengths): every stage inlined.
template <class P, class Acc, int DIR, int MODE0, bool FROM_SLOTS, int R0, int... Rs>
__device__ __forceinline__ void run_stages(const Acc& A, int N, int B, int Ns, uint32_t tw, const Consts<P>& k) {
  constexpr bool last = sizeof...(Rs) == 0;
  constexpr int MODE = MODE0 | ((DIR > 0 && last) ? kLast : 0);
  stage<P, Acc, R0, DIR, MODE, FROM_SLOTS>(A, N, B, Ns, tw, k);
  if constexpr (!last) run_stages<P, Acc, DIR, 0, !FROM_SLOTS, Rs...>(A, N, B, Ns * R0, tw + 16u * (uint32_t)(Ns * (R0 - 1)), k);
}

template <class P, class Acc, int... Rs>
__device__ __forceinline__ void pass_ct(const Acc& A, int N, int B, uint32_t tw, const Consts<P>& k,
                                        bool has_general) {
  constexpr bool even = (sizeof...(Rs) % 2) == 0;  // the spectrum lands in the slots
  run_stages<P, Acc, -1, kFirst, true, Rs...>(A, N, B, 1, tw, k);
  if (has_general) general_multiply<P, Acc>(A, B, even);
  run_stages<P, Acc, 1, kMul, even, Rs...>(A, N, B, 1, tw, k);
}

// Lengths with a compiled radix sequence (theta circles of 2 Ntheta = Nphi = LEN).
template <class P, class Acc, int LEN>
__device__ __forceinline__ void run_pass(const Acc& A, int N, int B, const Factors& f, uint32_t tw,
                                         const Consts<P>& k, bool g) {
  if constexpr (LEN == 32) pass_ct<P, Acc, 8, 4>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 64) pass_ct<P, Acc, 8, 8>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 96) pass_ct<P, Acc, 8, 4, 3>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 128) {
    // compensated FP32: 8, 4, 4 measured 9 % faster than 8, 8, 2 (smaller stage code); FP64 keeps
    // 8, 8, 2, which it runs without spilling
    if constexpr (std::is_same<P, DF>::value) pass_ct<P, Acc, 8, 4, 4>(A, LEN, B, tw, k, g);
    else pass_ct<P, Acc, 8, 8, 2>(A, LEN, B, tw, k, g);
  }
  else if constexpr (LEN == 192) pass_ct<P, Acc, 8, 8, 3>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 256) pass_ct<P, Acc, 8, 8, 4>(A, LEN, B, tw, k, g);
  else pass_rt<P, Acc>(A, N, B, f, tw, k, g);
}

// Each pass is its own function: its registers are allocated apart from the load/store code. HYB
// (hybrid fields: per-circle or per-ring tables, split multiplies of mixed pairs) is a compile-time
// flag, so that the other fields run code without those choices.
template <class P, int LEN, bool SPLIT = false, bool HYB = false>
__device__ __noinline__ void theta_pass_fn(ThetaAcc<P> TA, Factors f, uint32_t tw, Consts<P> K, int batch,
                                           bool has_general) {
  TA.template fix<LEN, SPLIT>();
  TA.hyb = HYB;
  for (int b0 = 0; b0 < TA.nseq; b0 += batch) {
    TA.b0 = b0;
    run_pass<P, ThetaAcc<P>, LEN>(TA, TA.M, min(batch, TA.nseq - b0), f, tw, K, HYB && has_general);
  }
}

template <class P, int LEN, bool HYB = false>
__device__ __noinline__ void phi_pass_fn(PhiAcc<P> PA, int npairs, bool has_general, Factors f, uint32_t tw,
                                         Consts<P> K, int batch) {
  PA.template fix<LEN>();
  PA.hyb = HYB;
  for (int b0 = 0; b0 < npairs; b0 += batch) {
    PA.b0 = b0;
    run_pass<P, PhiAcc<P>, LEN>(PA, PA.N, min(batch, npairs - b0), f, tw, K, has_general);
  }
}

template <class P, int LEN, bool HYB = false>
__device__ __noinline__ void phi_split_pass_fn(PhiSplitAcc<P> PA, int npairs, bool has_general, Factors f,
                                               uint32_t tw, Consts<P> K, int batch) {
  PA.template fix<LEN>();
  PA.hyb = HYB;
  for (int b0 = 0; b0 < npairs; b0 += batch) {
    PA.b0 = b0;
    run_pass<P, PhiSplitAcc<P>, LEN>(PA, PA.N, min(batch, npairs - b0), f, tw, K, has_general);
  }
}

// ------------------------------------------------------------------ spectral form (FP64)
//
// The theta pass is diagonal in the azimuthal mode m: shifting phi by pi multiplies mode m by
// (-1)^m, so the doubled circle of mode m is c[q] = X_q[m] (q < Ntheta) and (-1)^(a + m)
// X_{2 Ntheta - 1 - q}[m] (q >= Ntheta), X_j the phi spectrum of ring j. The filter
// F = Phi^-1 D T Phi (Sec. II.C, theta then phi) is then: one forward phi transform per ring, per
// mode m the theta filter T of the (anti)symmetric extension, the phi multiply D_m(j) =
// f(m, m_max(i, j)), one inverse phi transform; the transpose applies D before T. T runs on the
// Ntheta values X_j[m] themselves: with v_n = z_2n, v_{N-1-n} = z_{2n+1} (N = Ntheta, z_j = X_j[m],
// times (-1)^j for odd symmetry), V = FFT_N(v), U_l = a_l V_l + b_l V_{N-l} with a_l = g_l + g_{N-l},
// b_l = +-(g_l - g_{N-l}) e^{i pi l / N} (+ even, - odd; g_l = f(l) / (2 Ntheta)), u = IFFT_N(U)
// unnormalised, z'_2n = u_n, z'_{2n+1} = u_{N-1-n}: the cosine/sine (DCT-II/III, DST-II/III) pair
// written through a complex FFT of half the circle's length. The half spectra live in the rows
// (row stride Nphi + 2 holds Nphi/2 + 1 complex values).

// Theta filter of the modes m of the shell's half spectra: sequence b is mode m = b, its slots are
// the value pairs (2m, 2m + 1) of the rows (row index XOR-swizzled in groups of 8).
template <class P>
struct SpecAcc {
  using C = typename P::C;
  using T = typename P::T;
  struct Seq {
    int m;
    bool odd;      // (-1)^(a + m) = -1: antisymmetric extension
    bool general;  // unused (no split multiply)
  };
  uint32_t S, lin;
  int ld, N, N8, b0, parity, nh;
  bool phi_first;     // transpose: the phi multiply before the theta filter
  const void* gtab;   // phi multipliers f(|m|)/Nphi of this shell: [Ntheta][Nphi/2 + 1] (global)
  size_t gbase;

  __device__ __forceinline__ Seq seq(int b) const { return Seq{b, ((parity + b) & 1) != 0, false}; }
  __device__ __forceinline__ int seq_len() const { return N; }
  __device__ __forceinline__ uint32_t el(int row, int m) const { return S + (uint32_t)(row * ld + 2 * m) * 8u; }
  __device__ __forceinline__ int row_of(int n) const { return n < N / 2 ? 2 * n : 2 * (N - 1 - n) + 1; }
  __device__ __forceinline__ T phi_mult(int j, int m) const { return P::from_tab(gtab, gbase + (size_t)j * nh + m); }
  __device__ __forceinline__ C gather(const Seq& s, int n) const {
    const int j = row_of(n);
    C v = Cx<P>::neg_if(P::ld16(el(j, s.m)), s.odd && (j & 1));
    if (phi_first) v = Cx<P>::scale(v, phi_mult(j, s.m));
    return v;
  }
  __device__ __forceinline__ void scatter(const Seq& s, int n, C v) const {
    const int j = row_of(n);
    v = Cx<P>::neg_if(v, s.odd && (j & 1));
    if (!phi_first) v = Cx<P>::scale(v, phi_mult(j, s.m));
    P::st16(el(j, s.m), v);
  }
  __device__ __forceinline__ C slot_ld(const Seq& s, int n) const { return P::ld16(el(swz(n, N8), s.m)); }
  __device__ __forceinline__ void slot_st(const Seq& s, int n, C v) const { P::st16(el(swz(n, N8), s.m), v); }
  __device__ __forceinline__ T mult(const Seq&, int) const { return P::zero(); }  // not used
  __device__ __forceinline__ uint32_t lin_at(int b, int n) const {
    return lin + 16u * (uint32_t)((b - b0) * N + swz(n, N8));
  }
  __device__ __forceinline__ C lin_ld(int b, int n) const { return P::ld16(lin_at(b, n)); }
  __device__ __forceinline__ void lin_st(int b, int n, C v) const { P::st16(lin_at(b, n), v); }
};

// The inverse phi transform of a ring pair starts from the rings' half spectra: Z_m = X_j1[m] +
// i X_j2[m] for m <= Nphi/2, and conj(X_j1[N-m]) + i conj(X_j2[N-m]) above.
template <class P>
struct PhiHalfAcc : PhiAcc<P> {
  using C = typename P::C;
  using Seq = typename PhiAcc<P>::Seq;
  __device__ __forceinline__ C gather(const Seq& s, int m) const {
    const bool lo = m <= this->hN;
    const int mm = lo ? m : this->N - m;
    const C x1 = P::ld16(this->el(s.j1, 2 * mm)), x2 = P::ld16(this->el(s.j2, 2 * mm));
    return lo ? C{P::sub(x1.re, x2.im), P::add(x1.im, x2.re)} : C{P::add(x1.re, x2.im), P::sub(x2.re, x1.im)};
  }
};

// After the forward phi transform Z of x_j1 + i x_j2 (in the slots or the scratch): the half
// spectra X_j1[m] = (Z_m + conj Z_{N-m}) / 2 and X_j2[m] = (Z_m - conj Z_{N-m}) / (2i), m = 0 .. N/2,
// over the rows. A spectrum in the slots (the rows themselves) is first moved to the scratch, so
// that no write of the split lands on a value still to be read.
template <class P>
__device__ void split_spectra(const PhiAcc<P>& A, int B, bool in_slots) {
  using C = typename P::C;
  const int N = A.N, nh = N / 2 + 1;
  if (in_slots) {
    for (int w = threadIdx.x; w < B * N; w += blockDim.x) {
      const int bl = w / N, n = w - bl * N;
      const int b = A.b0 + bl;
      A.lin_st(b, n, A.slot_ld(A.seq(b), n));
    }
    __syncthreads();
  }
  for (int base = 0; base < B * nh; base += blockDim.x) {
    const int w = base + threadIdx.x;
    const bool act = w < B * nh;
    typename PhiAcc<P>::Seq sq{};
    int m = 0;
    C x1{}, x2{};
    if (act) {
      const int bl = w / nh;
      const int b = A.b0 + bl;
      m = w - bl * nh;
      sq = A.seq(b);
      const C zm = A.lin_ld(b, m), zn = A.lin_ld(b, (N - m) % N);
      x1 = C{P::half(P::add(zm.re, zn.re)), P::half(P::sub(zm.im, zn.im))};
      x2 = C{P::half(P::add(zm.im, zn.im)), P::half(P::sub(zn.re, zm.re))};
    }
    __syncthreads();
    if (act) {
      P::st16(A.el(sq.j1, 2 * m), x1);
      P::st16(A.el(sq.j2, 2 * m), x2);
    }
    __syncthreads();
  }
}

// Before an inverse phi transform with an odd number of stages: Z_m (as PhiHalfAcc::gather forms it)
// for every m into the scratch, so that the stages run scratch -> slots -> ... and the last one,
// which writes the rows, reads the scratch (a last stage reading the slots, the rows themselves,
// would race with its own writes).
template <class P>
__device__ void merge_spectra(const PhiHalfAcc<P>& A, int B) {
  const int N = A.N;
  for (int w = threadIdx.x; w < B * N; w += blockDim.x) {
    const int bl = w / N, m = w - bl * N;
    const int b = A.b0 + bl;
    A.lin_st(b, m, A.gather(A.seq(b), m));
  }
  __syncthreads();
}

// The theta filter between the forward and inverse length-N transforms of each mode in the batch:
// U_l = a_l V_l + b_l V_{N-l}, U_{N-l} = a_l V_{N-l} + conj(b_l) V_l (pairs l <= N/2). g: the theta
// multipliers f(l)/(2 Ntheta), l = 0 .. N (shared); e: e^{i pi l / N}, l < N (shared).
template <class P>
__device__ void dct_multiply(const SpecAcc<P>& A, int B, bool in_slots, uint32_t g, uint32_t e) {
  using C = typename P::C;
  using T = typename P::T;
  const int N = A.N, half = N / 2;
  for (int base = 0; base < B * (half + 1); base += blockDim.x) {
    const int w = base + threadIdx.x;
    const bool act = w < B * (half + 1);
    typename SpecAcc<P>::Seq sq{};
    int l = 0, ln = 0, b = 0;
    C u1{}, u2{};
    if (act) {
      const int bl = w / (half + 1);
      b = A.b0 + bl;
      l = w - bl * (half + 1);
      ln = (N - l) % N;
      sq = A.seq(b);
      const C v1 = in_slots ? A.slot_ld(sq, l) : A.lin_ld(b, l);
      const C v2 = in_slots ? A.slot_ld(sq, ln) : A.lin_ld(b, ln);
      const T gl = P::ld8(g + 8u * (uint32_t)l), gn = P::ld8(g + 8u * (uint32_t)(N - l));
      const T a = P::add(gl, gn);
      const T d = sq.odd ? P::sub(gn, gl) : P::sub(gl, gn);
      const C ez = P::ld16(e + 16u * (uint32_t)l);
      const C bc{P::mul(d, ez.re), P::mul(d, ez.im)};
      u1 = Cx<P>::add(Cx<P>::scale(v1, a), P::cmul(v2, bc));
      u2 = Cx<P>::add(Cx<P>::scale(v2, a), P::cmul(v1, Cx<P>::conj(bc)));
    }
    __syncthreads();
    if (act) {
      if (in_slots) {
        A.slot_st(sq, l, u1);
        if (ln != l) A.slot_st(sq, ln, u2);
      } else {
        A.lin_st(b, l, u1);
        if (ln != l) A.lin_st(b, ln, u2);
      }
    }
    __syncthreads();
  }
}

// Forward stages of a batch (first stage gathers); true if the spectrum lands in the slots.
// Compile-time radix sequences for the FP64 128-point (8, 8, 2) and 64-point (8, 8) transforms,
// else the plan's factorisation f.
template <class P, class Acc, int NLEN>
__device__ __forceinline__ bool fwd_stages(const Acc& A, int N, int B, const Factors& f, uint32_t tw,
                                           const Consts<P>& k) {
  if constexpr (NLEN == 128) {
    run_stages<P, Acc, -1, kFirst, true, 8, 8, 2>(A, N, B, 1, tw, k);
    return false;
  } else if constexpr (NLEN == 64) {
    run_stages<P, Acc, -1, kFirst, true, 8, 8>(A, N, B, 1, tw, k);
    return true;
  } else {
    int Ns = 1;
    uint32_t ts = tw;
    for (int s = 0; s < f.nst; ++s) {
      const int R = f.radix[s];
      if (s == 0) stage_r<P, Acc, -1, kFirst>(R, A, N, B, Ns, ts, k, true);
      else stage_r<P, Acc, -1, 0>(R, A, N, B, Ns, ts, k, (s & 1) == 0);
      ts += 16u * (uint32_t)(Ns * (R - 1));
      Ns *= R;
    }
    return (f.nst & 1) == 0;
  }
}

// Inverse stages of a batch: the first stage gathers (FIRST) or reads the slots/scratch holding the
// forward result (the slots when `slots`); the last stage scatters.
template <class P, class Acc, int NLEN, bool FIRST>
__device__ __forceinline__ void inv_stages(const Acc& A, int N, int B, const Factors& f, uint32_t tw,
                                           const Consts<P>& k, bool slots) {
  constexpr int M0 = FIRST ? kFirst : 0;
  if constexpr (NLEN == 128) {
    if (FIRST || slots) run_stages<P, Acc, 1, M0, true, 8, 8, 2>(A, N, B, 1, tw, k);
    else run_stages<P, Acc, 1, M0, false, 8, 8, 2>(A, N, B, 1, tw, k);
  } else if constexpr (NLEN == 64) {
    if (FIRST || slots) run_stages<P, Acc, 1, M0, true, 8, 8>(A, N, B, 1, tw, k);
    else run_stages<P, Acc, 1, M0, false, 8, 8>(A, N, B, 1, tw, k);
  } else {
    int Ns = 1;
    uint32_t ts = tw;
    for (int s = 0; s < f.nst; ++s) {
      const int R = f.radix[s];
      const bool first = s == 0, last = s == f.nst - 1;
      const bool from_slots = (FIRST || slots) ? (s & 1) == 0 : (s & 1) == 1;
      if (first && last) stage_r<P, Acc, 1, M0 | kLast>(R, A, N, B, Ns, ts, k, from_slots);
      else if (first) stage_r<P, Acc, 1, M0>(R, A, N, B, Ns, ts, k, from_slots);
      else if (last) stage_r<P, Acc, 1, kLast>(R, A, N, B, Ns, ts, k, from_slots);
      else stage_r<P, Acc, 1, 0>(R, A, N, B, Ns, ts, k, from_slots);
      ts += 16u * (uint32_t)(Ns * (R - 1));
      Ns *= R;
    }
  }
}

// The spectral form on a shell whose theta pass is active (every ring pair in PA's list): forward
// phi transforms and half spectra; per mode the theta filter and the phi multiply; inverse phi
// transforms. tw_sp: the length-Ntheta stage twiddles, then e^{i pi l / Ntheta} (Ntheta entries
// each); g_th: the theta multipliers.
template <class P, int LEN>
__device__ __noinline__ void spectral_fn(PhiAcc<P> PA, SpecAcc<P> SA, int npairs, Factors fph, Factors fsp,
                                         uint32_t tw_ph, uint32_t tw_sp, uint32_t g_th, Consts<P> K, int batch_ph,
                                         int batch_sp) {
  PA.template fix<LEN>();
  const int Nph = PA.N, Nth = SA.N;
  for (int b0 = 0; b0 < npairs; b0 += batch_ph) {
    PA.b0 = b0;
    const int B = min(batch_ph, npairs - b0);
    const bool in_slots = fwd_stages<P, PhiAcc<P>, LEN>(PA, Nph, B, fph, tw_ph, K);
    split_spectra<P>(PA, B, in_slots);
  }
  const int nm = Nph / 2 + 1;
  const uint32_t dct = tw_sp + 16u * (uint32_t)Nth;
  for (int b0 = 0; b0 < nm; b0 += batch_sp) {
    SA.b0 = b0;
    const int B = min(batch_sp, nm - b0);
    const bool in_slots = fwd_stages<P, SpecAcc<P>, LEN / 2>(SA, Nth, B, fsp, tw_sp, K);
    dct_multiply<P>(SA, B, in_slots, g_th, dct);
    inv_stages<P, SpecAcc<P>, LEN / 2, false>(SA, Nth, B, fsp, tw_sp, K, in_slots);
  }
  // inverse phi transforms: the last stage must read the scratch (its writes go to the rows), so an
  // odd number of stages starts from the scratch (merge_spectra), an even one gathers directly
  PhiHalfAcc<P> HA;
  static_cast<PhiAcc<P>&>(HA) = PA;
  const bool odd_stages = LEN == 128 ? true : (fph.nst & 1) != 0;
  for (int b0 = 0; b0 < npairs; b0 += batch_ph) {
    HA.b0 = b0;
    const int B = min(batch_ph, npairs - b0);
    if (odd_stages) {
      merge_spectra<P>(HA, B);
      inv_stages<P, PhiHalfAcc<P>, LEN, false>(HA, Nph, B, fph, tw_ph, K, false);
    } else {
      inv_stages<P, PhiHalfAcc<P>, LEN, true>(HA, Nph, B, fph, tw_ph, K, true);
    }
  }
}

// ------------------------------------------------------------------ kernel

template <class P>
struct Layout {
  unsigned char* buf;  // the shell
  uint32_t lin;        // FFT scratch
  uint32_t ov, tw_th, tw_ph, g_th;
  int2* pairs;
  int* misc;               // [0] pair count, [1] general flag, [2] block max exponent, [3] active rows,
                           // hybrid fields: [4] mixed circle pairs, [5] some circle fired, [6] scratch
  unsigned char* rowact;   // rows that are transformed (1) or passed through unchanged (0)
  unsigned short* arow;    // the transformed rows, ascending
  unsigned char* circ;     // hybrid fields: detector flags of the theta circles [Nphi/2],
  unsigned char* ring;     //   of the phi rings [Ntheta],
  unsigned char* thsel;    //   and the table choice of each theta sequence [(Nphi/2 + 1)/2]
  uint32_t bar;            // mbarrier of the shell's bulk copies (8 bytes), then the wait's outcome
  int* wait_flag;          //   (4 bytes)
};

// Scratch for one batch: batch_th theta sequences (2 Ntheta slots each) or batch_ph phi pairs
// (Nphi slots each).
__host__ __device__ __forceinline__ size_t scratch_bytes(const ShellArgs2& A) {
  const size_t th = (size_t)A.batch_th * 2 * A.Nth;
  const size_t ph = (size_t)A.batch_ph * A.Nph;
  return 16 * (th > ph ? th : ph);
}

template <class P>
__device__ Layout<P> carve(const ShellArgs2& A, unsigned char* base) {
  Layout<P> L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off = (off + bytes + 15) / 16 * 16;
    return p;
  };
  const size_t shell_bytes = 8 * (size_t)A.Nth * A.ldS;
  L.buf = take(shell_bytes);
  L.lin = saddr(take(scratch_bytes(A)));
  L.ov = saddr(take(16 * (size_t)max(2 * A.Nth, A.Nph)));
  L.tw_th = saddr(take(16 * 2 * (size_t)A.Nth));
  L.tw_ph = saddr(take(16 * (size_t)A.Nph));
  L.g_th = saddr(take(16 * (size_t)(A.Nth + 1)));  // two rows: a hybrid field's Gaussian one second
  L.pairs = reinterpret_cast<int2*>(take(sizeof(int2) * (size_t)(A.Nth / 2 + 1)));
  L.misc = reinterpret_cast<int*>(take(sizeof(int) * 8));
  L.rowact = take((size_t)A.Nth);
  L.arow = reinterpret_cast<unsigned short*>(take(sizeof(unsigned short) * (size_t)A.Nth));
  L.circ = take((size_t)(A.Nph / 2 + A.Nth + (A.Nph / 2 + 1) / 2));
  L.ring = L.circ + A.Nph / 2;
  L.thsel = L.ring + A.Nth;
  unsigned char* b = take(16);
  L.bar = saddr(b);
  L.wait_flag = reinterpret_cast<int*>(b + 8);
  return L;
}

template <class P>
__device__ __forceinline__ typename P::T to_real(double x, int E);
template <>
__device__ __forceinline__ double to_real<F64>(double x, int) { return x; }
template <>
__device__ __forceinline__ df to_real<DF>(double x, int E) { return df_from_double(x, E); }

template <class P>
__device__ __forceinline__ double from_real(typename P::T x, int E);
template <>
__device__ __forceinline__ double from_real<F64>(double x, int) { return x; }
template <>
__device__ __forceinline__ double from_real<DF>(df x, int E) { return df_to_double(x, E); }

// Shell s of the launch in i-major order over the launched fields (the fields of one radius run
// together, so their multiplier rows stay in L2); returns the element offset of the shell in the
// [var][shell] layout of the whole state.
__device__ __forceinline__ size_t shell_offset(const ShellArgs2& A, const LaunchIO& io, int s, int* v, int* i) {
  *i = s / io.var_count;
  *v = io.var_begin + (s - *i * io.var_count);
  return ((size_t)*v * A.Nr + *i) * (size_t)A.Nth * A.Nph;
}

// In-place plain FP64 calls move only the rows a pass transforms: the others already hold their
// result in memory. Compiled in for the 128-point length (whose register budget has room for it).
template <int LEN>
__device__ __forceinline__ bool in_place_sparse(const LaunchIO& io) {
  return LEN == 128 && io.in == io.out && !io.is_f32 && io.async_ok && io.map_in == kMapNone &&
         io.map_out == kOutNone && !io.hybrid;  // hybrid fields: every row may be transformed
}

// The shell's bulk copies (TMA engine), issued by warp 0: one per row (Nphi values, contiguous in
// the state) into the padded rows of the buffer (row stride Nphi + 2: 16-byte aligned, Nphi even),
// all completing on the shell's mbarrier.
template <int LEN>
__device__ __forceinline__ void issue_shell_copies(const ShellArgs2& A, const LaunchIO& io, int s,
                                                   const unsigned char* buf, uint32_t bar) {
  int v, i;
  const double* src = static_cast<const double*>(io.in) + shell_offset(A, io, s, &v, &i);
  const int Nth = LEN ? LEN / 2 : A.Nth, Nph = LEN ? LEN : A.Nph, ldS = LEN ? LEN + 2 : A.ldS;
  const uint32_t lane = threadIdx.x & 31, dst = saddr(buf), row_bytes = 8u * (uint32_t)Nph;
  if (lane == 0) bar_expect(bar, row_bytes * (uint32_t)Nth);
  __syncwarp();
  for (int row = (int)lane; row < Nth; row += 32)
    bulk_g2s(dst + (uint32_t)(row * ldS) * 8u, src + (size_t)row * Nph, row_bytes, bar);
}

// Staging policy: the FP64 form stages its shells by bulk copies; the compensated-FP32 form by
// 16-byte cp.async from every thread, which measured faster there (its two CTAs per SM overlap the
// copies with each other's arithmetic either way).
template <class P>
__host__ __device__ constexpr bool bulk_staging() {
  return std::is_same<P, F64>::value;
}

// The shell's copies by 16-byte cp.async from every thread into the padded rows (waited for with
// cp.async.wait_group).
template <int LEN>
__device__ __forceinline__ void issue_shell_async(const ShellArgs2& A, const LaunchIO& io, int s, unsigned char* buf) {
  int v, i;
  const double* src = static_cast<const double*>(io.in) + shell_offset(A, io, s, &v, &i);
  const int Nth = LEN ? LEN / 2 : A.Nth, Nph = LEN ? LEN : A.Nph, ldS = LEN ? LEN + 2 : A.ldS;
  const int half = Nph / 2, total = Nth * half;
  const uint32_t dst = saddr(buf);
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    const int row = c / half, k2 = c - row * half;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (uint32_t)(row * ldS + 2 * k2) * 8u),
                 "l"(src + (size_t)row * Nph + 2 * k2)
                 : "memory");
  }
}

// ------------------------------------------------------------------ hybrid filter: shock detector

// x 2^-E as FP32 for the detector's screen, E = emax - 1023 with emax the largest exponent field of
// the shell's finite values (so |x 2^-E| < 2), from the high word of x alone: the significand keeps
// its 20 leading bits (relative error below 2^-20), values under 2^-120 on that scale become 0.
// Subnormal, infinite and NaN inputs give NaN, which sends their cells to the exact decision;
// zero converts exactly.
__device__ __forceinline__ float screen_value(double x, int emax) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int fe = e - emax + 127;  // FP32 biased exponent on the shell's scale
  const float v = __uint_as_float((hi & 0x80000000u) | ((unsigned)fe << 23) | ((hi & 0xfffffu) << 3));
  if ((unsigned)(e - 1) >= 0x7feu)  // zero, subnormal, infinite or NaN
    return (u << 1) == 0ull ? 0.0f : __int_as_float(0x7fffffff);
  return fe >= 7 ? v : 0.0f;
}

// The same conversion for the column walk, for shells whose values are all zero or normal and whose
// emax is at least 128: |x| is clamped to the scale's 2^-120 floor (floor_a = (emax - 120) << 20 on
// the high word without its sign; an absolute change below 2^-119, like the flush above), then the
// exponent is rebased (adj = (emax - 127) << 20) and moved into place.
__device__ __forceinline__ float screen_value_walk(double x, unsigned floor_a, unsigned adj) {
  const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32);
  const unsigned a = max(hi & 0x7fffffffu, floor_a);
  return __uint_as_float(((a - adj) << 3) | (hi & 0x80000000u));
}

// Jameson's sigma >= 0.95 for the cell b between a and c, in FP64 with round-to-nearest, operation
// for operation: num = |(a + c) - 2 b|, den = ((|a| + |c|) + 2 |b|) + eps, num / den >= 0.95. Out of
// line, so that the compiler cannot evaluate it ahead of the screen that rarely needs it (the FP64
// pipe is slow on this GPU). A template only to give it one definition per translation unit.
template <int = 0>
__device__ __noinline__ bool jameson_exact(double a, double b, double c, double eps) {
  const double num = fabs(__dsub_rn(__dadd_rn(a, c), __dmul_rn(2.0, b)));
  const double den = __dadd_rn(__dadd_rn(__dadd_rn(fabs(a), fabs(c)), __dmul_rn(2.0, fabs(b))), eps);
  return __ddiv_rn(num, den) >= 0.95;
}

// The same decision screened in FP32 on the shell's scale: 1 fires, 0 does not, -1 undecided.
// Error budget: the inputs carry relative errors below 2^-20, so num and den move by less than
// 2^-20 D each (D = |a| + 2|b| + |c| <= den), and their four FP32 roundings add less than 2^-22 den;
// with den_f >= 2^-80 the flushed values and the rounding of eps do not count. Hence
// |num_f - sigma den_f| < 2.3e-6 den_f, and s = num_f - 0.95 den_f (one FMA, 0.95f within 1.2e-8
// of 0.95) decides every cell with |sigma - 0.95| > 4e-6 exactly as the FP64 expression does.
// Cells inside the band, or with a NaN (flagged) input, are undecided and take that expression.
__device__ __forceinline__ int jameson_screen(float af, float bf, float cf, float epsf) {
  const float num = fabsf(__fmaf_rn(-2.0f, bf, __fadd_rn(af, cf)));
  const float den = __fadd_rn(__fmaf_rn(2.0f, fabsf(bf), __fadd_rn(fabsf(af), fabsf(cf))), epsf);
  const float sv = __fmaf_rn(-0.95f, den, num), m = 4e-6f * den;
  if (den >= 0x1p-80f) {
    if (sv >= m) return 1;
    if (sv < -m) return 0;
  }
  return -1;
}

// Where the detector finds a shell's FP64 values. DetShell: the whole shell in this CTA (row stride
// lds, W = Nphi columns, periodic rings). The cluster kernel's DetHalf (defined with it) holds half
// of the meridians and reads its rings' other half from the peer CTA.
template <int LEN>
struct DetShell {
  static constexpr bool kPair = false;
  uint32_t S;
  int nth, w, ld;
  __device__ __forceinline__ int Nth() const { return LEN ? LEN / 2 : nth; }
  __device__ __forceinline__ int W() const { return LEN ? LEN : w; }
  __device__ __forceinline__ int lds() const { return LEN ? LEN + 2 : ld; }
  __device__ __forceinline__ double at(int j, int c) const { return F64::ld8(S + 8u * (uint32_t)(j * lds() + c)); }
  // the phi neighbour of column c on row j (dir = -1 left, +1 right)
  __device__ __forceinline__ double nbr(int j, int c, int dir) const {
    c += dir;
    return at(j, c < 0 ? W() - 1 : (c == W() ? 0 : c));
  }
};

// Jameson's shock detector of the hybrid filter (Sec. II.C) on the FP64 values the geometry G holds
// (W columns, W/2 circles: column c and c + W/2 are the two meridians of circle c < W/2): ring[j] = 1
// if some cell of phi ring j has sigma >= 0.95, circ[c] = 1 likewise for theta circle c (the values
// across a pole with the parity sign). misc[5] = 1 if some circle fired; misc[6], misc[7] are
// scratch. For a CTA pair both CTAs screen on one scale and leave with the ring flags and misc[5]
// combined over the pair. Called by every thread of the CTA; the caller synchronises afterwards.
// When W is a multiple of 32 and at most the block size, thread t walks column t mod W down one band
// of rows: each value is read and converted once, the theta neighbours are the previous and the next
// row of the walk, and the phi neighbours come from the adjacent lanes (a warp holds 32 consecutive
// columns of one band; its edge lanes read theirs); it only screens. Without the walk (other W,
// values that are subnormal or not finite, emax < 128), or when the screen left a cell undecided,
// every cell reads its four neighbours and undecided cells take the FP64 expression.
template <class G>
__device__ __noinline__ void detect_shell(const G g, bool odd, double eps, float eps_m, int eps_p, unsigned char* circ,
                                          unsigned char* ring, int* misc) {
  const int Nth = g.Nth(), W = g.W(), h = W / 2;
  const unsigned long long flip = odd ? 0x8000000000000000ull : 0ull;
  auto across = [&](double x) { return __longlong_as_double(__double_as_longlong(x) ^ flip); };
  for (int n = threadIdx.x; n < h + Nth; n += blockDim.x) circ[n] = 0;  // circ, then ring
  if (threadIdx.x == 0) {
    misc[5] = 0;
    misc[6] = 0;
  }
  const int bands = (W & 31) == 0 ? (int)blockDim.x / W : 0;
  const int t = threadIdx.x, k = bands ? t % W : 0, band = bands ? t / W : 0;
  const int j0 = band < bands ? band * Nth / bands : 0, j1 = band < bands ? (band + 1) * Nth / bands : 0;
  // the largest exponent field of the finite values, and whether any value is subnormal or not finite
  unsigned em = 0;
  bool special = false;
  auto take = [&](double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
    special |= e == 0x7ffu || (e == 0u && (u << 1) != 0ull);
    if (e != 0x7ffu) em = max(em, e);
  };
  if (bands) {
    for (int j = j0; j < j1; ++j) take(g.at(j, k));
  } else {
    for (int n = threadIdx.x; n < Nth * W; n += blockDim.x) take(g.at(n / W, n % W));
  }
  em = __reduce_max_sync(0xffffffffu, em);
  __syncthreads();  // flags and misc cleared
  if ((threadIdx.x & 31) == 0) atomicMax(&misc[6], (int)em);
  bool any_special = __syncthreads_or(special) != 0;
  int emax = misc[6];
  if constexpr (G::kPair) {
    // one scale for the pair: the edge values come from the peer
    if (threadIdx.x == 0) misc[7] = any_special ? 1 : 0;
    g.pair_sync();  // also: the peer's values are in its shared memory
    emax = max(emax, g.peer_int(&misc[6]));
    any_special |= g.peer_int(&misc[7]) != 0;
  }
  const float epsf = ldexpf(eps_m, eps_p + 1023 - emax);  // eps on the scale, in FP32 (0 or inf at the ends)
  bool fired = false, undecided = false;
  if (bands && !any_special && emax >= 128) {
    const unsigned floor_a = (unsigned)(emax - 120) << 20, adj = (unsigned)(emax - 127) << 20;
    if (band < bands) {  // whole warps
      const int lane = t & 31, ko = k < h ? k + h : k - h;  // ko: the column across the pole
      const int c = k < h ? k : k - h;
      // the phi neighbour a lane cannot take from the adjacent lane: left for lane 0, right for 31
      const int dir = lane == 0 ? -1 : 1;
      float upf = screen_value_walk(j0 > 0 ? g.at(j0 - 1, k) : across(g.at(0, ko)), floor_a, adj);
      float cuf = screen_value_walk(g.at(j0, k), floor_a, adj);
#pragma unroll 2
      for (int j = j0; j < j1; ++j) {
        const float dnf = screen_value_walk(j < Nth - 1 ? g.at(j + 1, k) : across(g.at(Nth - 1, ko)), floor_a, adj);
        const float ef = screen_value_walk(g.nbr(j, k, dir), floor_a, adj);
        int d = jameson_screen(upf, cuf, dnf, epsf);
        undecided |= d < 0;
        if (d > 0) {
          circ[c] = 1;
          fired = true;
        }
        const float lsh = __shfl_up_sync(0xffffffffu, cuf, 1), rsh = __shfl_down_sync(0xffffffffu, cuf, 1);
        d = jameson_screen(lane == 0 ? ef : lsh, cuf, lane == 31 ? ef : rsh, epsf);
        undecided |= d < 0;
        if (d > 0) ring[j] = 1;
        upf = cuf;
        cuf = dnf;
      }
    }
  } else {
    undecided = true;
  }
  // a shell with an undecided cell anywhere (rare) takes the cell-by-cell pass below, which repeats
  // every decision (the same screen) and settles the undecided ones with the FP64 expression
  if (__syncthreads_or(undecided)) {
    for (int n = threadIdx.x; n < Nth * W; n += blockDim.x) {
      const int j = n / W, kk = n - j * W;
      const int ko = kk < h ? kk + h : kk - h;
      const double b = g.at(j, kk);
      const double pa = g.nbr(j, kk, -1), pc = g.nbr(j, kk, 1);
      const double ta = j > 0 ? g.at(j - 1, kk) : across(g.at(0, ko));
      const double tc = j < Nth - 1 ? g.at(j + 1, kk) : across(g.at(Nth - 1, ko));
      const float bf = screen_value(b, emax);
      int d = jameson_screen(screen_value(pa, emax), bf, screen_value(pc, emax), epsf);
      if (d < 0) d = jameson_exact(pa, b, pc, eps);
      if (d) ring[j] = 1;
      d = jameson_screen(screen_value(ta, emax), bf, screen_value(tc, emax), epsf);
      if (d < 0) d = jameson_exact(ta, b, tc, eps);
      if (d) {
        circ[kk < h ? kk : kk - h] = 1;
        fired = true;
      }
    }
  }
  if (__any_sync(0xffffffffu, fired) && (threadIdx.x & 31) == 0) misc[5] = 1;
  if constexpr (G::kPair) {
    // the pair's ring flags and "a circle fired" are the union of both halves (OR is idempotent,
    // so reading the peer's flags while it ORs ours in is harmless)
    g.pair_sync();  // both halves' flags are final; the peer's values are not read after this
    for (int j = threadIdx.x; j < Nth; j += blockDim.x)
      if (g.peer_u8(ring + j)) ring[j] = 1;
    if (threadIdx.x == 0 && g.peer_int(&misc[5])) misc[5] = 1;
  }
}

// HYB: the kernel variant for launches with hybrid fields (the other variant has none of their code).
template <class P, int LEN, bool HYB, bool SPEC = false>
__device__ void filter_shell(const ShellArgs2& A, const LaunchIO& io, const Layout<P>& L, unsigned char* buf, int s,
                             const Consts<P>& K, bool copies_issued) {
  constexpr bool dfp = std::is_same<P, DF>::value;
  // the shell's bulk copies (issued by the kernel, or below by an in-place call) are awaited once,
  // where the values are first needed
  bool pending = copies_issued;
  auto arrived = [&]() -> bool {
    if (!pending) return true;
    pending = false;
    return wait_copies(A.status, L.bar, L.wait_flag);
  };
  int v, i;
  const size_t off = shell_offset(A, io, s, &v, &i);
  const VarInfo vi = A.var[v];
  // compile-time sizes for the fixed lengths (divisions by Nphi become shifts or multiplies)
  const int Nth = LEN ? LEN / 2 : A.Nth, Nph = LEN ? LEN : A.Nph, ld = LEN ? LEN + 2 : A.ldS;
  const int npts = Nth * Nph;
  double* Sd = reinterpret_cast<double*>(buf);

  // FP32 or unaligned input: synchronous load (8 loads in flight per thread), as FP64 in the buffer
  if (io.is_f32 || !io.async_ok) {
    const float* srcf = static_cast<const float*>(io.in) + off;
    const double* srcd = static_cast<const double*>(io.in) + off;
    constexpr int kBatch = 8;
    for (int n0 = 0; n0 < npts; n0 += kBatch * blockDim.x) {
      double xv[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int n = n0 + u * blockDim.x + threadIdx.x;
        xv[u] = n < npts ? (io.is_f32 ? (double)__ldcs(srcf + n) : __ldcs(srcd + n)) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int n = n0 + u * blockDim.x + threadIdx.x;
        if (n < npts) Sd[(n / Nph) * ld + n % Nph] = xv[u];
      }
    }
    __syncthreads();
  }
  // per-shell tables: theta multipliers, phi ring pairs, rows that will be transformed
  const double lmax = A.lmax[vi.cls * A.Nr + i];
  const bool gauss = vi.kind == SPH_FILTER_GAUSS;
  const bool hyb = HYB && vi.kind == SPH_FILTER_HYBRID;
  const size_t gth_base = ((size_t)vi.cls * A.Nr + i) * (Nth + 1);
  const size_t gth_alt = ((size_t)vi.alt_cls * A.Nr + i) * (Nth + 1);
  // theta multipliers: 8-byte table entries copied as they are (FP64, or an FP32 pair); a hybrid
  // field's Gaussian row follows its exponential one
  for (int n = threadIdx.x; n < (hyb ? 2 : 1) * (Nth + 1); n += blockDim.x) {
    const size_t t = n <= Nth ? gth_base + n : gth_alt + (n - (Nth + 1));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(L.g_th + 8u * n),
                 "l"(static_cast<const unsigned char*>(A.g_th) + 8 * t)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (hyb) {
    // a hybrid field's choices come from the whole FP64 shell: wait for it, run the detector
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!arrived()) return;
    __syncthreads();
    DetShell<LEN> geo;
    geo.S = saddr(buf);
    geo.nth = Nth;
    geo.w = Nph;
    geo.ld = ld;
    detect_shell(geo, vi.parity != 0, A.eps, A.eps_m, A.eps_p, L.circ, L.ring, L.misc);
    __syncthreads();
  }
  const bool theta_on = gauss || lmax < (double)Nth || (hyb && L.misc[5] != 0);
  for (int j = threadIdx.x; j < Nth; j += blockDim.x) L.rowact[j] = theta_on ? 1 : 0;
  const uint8_t* ring_info = A.ring_info + ((size_t)vi.cls * A.Nr + i) * Nth;
  const uint8_t* ring_alt = A.ring_info + ((size_t)vi.alt_cls * A.Nr + i) * Nth;
  __syncthreads();
  if (threadIdx.x < 32) {
    // active ring pairs in ascending j, compacted by one warp (ballot + prefix count)
    const unsigned lane = threadIdx.x;
    int np = 0, gen = 0;
    for (int j0 = 0; j0 < (Nth + 1) / 2; j0 += 32) {
      const int j = j0 + (int)lane, jj = Nth - 1 - j;
      const bool in = j < (Nth + 1) / 2;
      const uint8_t a = in ? ring_info[j] : 0, b = in ? ring_info[jj] : 0;
      // hybrid field: a ring whose detector fired takes the Gaussian table (never the identity)
      const int fa = (hyb && in) ? L.ring[j] : 0, fb = (hyb && in) ? L.ring[jj] : 0;
      // bit 0: ring active; the spectral form transforms every ring of a shell with a theta pass
      const bool act = ((a | b) & 1) != 0 || fa || fb || (SPEC && theta_on && in);
      // the multipliers of j and its mirror differ: different tables, or one table whose cutoffs
      // differ beyond rounding (bit 1)
      const int g = fa != fb ? 1 : ((fa ? (in ? ring_alt[j] : 0) : a) >> 1) & 1;
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if (act) {
        const int pos = np + __popc(m & ((1u << lane) - 1u));
        L.rowact[j] = L.rowact[jj] = 1;
        L.pairs[pos] = jj == j ? make_int2(j | (fa << 29), -1) : make_int2(j | (g << 30) | (fa << 29) | (fb << 28), jj);
      }
      gen |= __any_sync(0xffffffffu, act && jj != j && g) ? 1 : 0;
      np += __popc(m);
    }
    // the transformed rows, compacted (rowact is final for this warp after the sync)
    __syncwarp();
    int na = 0;
    for (int j0 = 0; j0 < Nth; j0 += 32) {
      const int j = j0 + (int)lane;
      const bool act = j < Nth && L.rowact[j];
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if (act) L.arow[na + __popc(m & ((1u << lane) - 1u))] = (unsigned short)j;
      na += __popc(m);
    }
    // hybrid field: table of each theta sequence (circles 2b, 2b+1): 0 exponential, 1 Gaussian,
    // 2 one of each (split multiply); a lone last circle counts twice
    int gth = 0;
    if (hyb) {
      const int h = Nph / 2, nseq = (h + 1) / 2;
      for (int b0 = 0; b0 < nseq; b0 += 32) {
        const int b = b0 + (int)lane;
        int t = 0;
        if (b < nseq) {
          const int c1 = L.circ[2 * b], c2 = 2 * b + 1 < h ? L.circ[2 * b + 1] : c1;
          t = c1 == c2 ? c1 : 2;
          L.thsel[b] = (unsigned char)t;
        }
        gth |= __any_sync(0xffffffffu, t == 2) ? 1 : 0;
      }
    }
    if (lane == 0) {
      L.misc[0] = np;
      L.misc[1] = gen;
      L.misc[3] = na;
      L.misc[4] = gth;
    }
  }
  if (in_place_sparse<LEN>(io)) {
    __syncthreads();  // the active-row list is in place
    const int na = L.misc[3];
    if (na == 0) {  // nothing to transform: the shell already holds its result
      asm volatile("cp.async.wait_all;" ::: "memory");
      return;
    }
    // copies of the transformed rows only (bulk: warp 0, one per row)
    if (!bulk_staging<P>()) {
      const double* src = static_cast<const double*>(io.in) + off;
      const uint32_t dst = saddr(buf);
      for (int c = threadIdx.x; c < na * (Nph / 2); c += blockDim.x) {
        const int row = (int)L.arow[c / (Nph / 2)], k2 = c % (Nph / 2);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (uint32_t)(row * ld + 2 * k2) * 8u),
                     "l"(src + (size_t)row * Nph + 2 * k2)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else if (threadIdx.x < 32) {
      const double* src = static_cast<const double*>(io.in) + off;
      const uint32_t dst = saddr(buf), row_bytes = 8u * (uint32_t)Nph;
      if (threadIdx.x == 0) bar_expect(L.bar, row_bytes * (uint32_t)na);
      __syncwarp();
      for (int c = (int)threadIdx.x; c < na; c += 32) {
        const int row = (int)L.arow[c];
        bulk_g2s(dst + (uint32_t)(row * ld) * 8u, src + (size_t)row * Nph, row_bytes, L.bar);
      }
    }
    pending = bulk_staging<P>();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!arrived()) return;
  __syncthreads();  // tables, twiddles, pair list and the shell's values are in place

  // input map on every value; block exponent and conversion to the working precision (in place)
  // only on the rows that are transformed: the others are stored back as they were loaded
  unsigned emax = 0;
  const int nact = L.misc[3];
  if (io.map_in == kMapTanh) {
    for (int n = threadIdx.x; n < npts; n += blockDim.x) {
      const int jrow = n / Nph;
      const int o = jrow * ld + n % Nph;
      const double x = map_tanh<P>(Sd[o]);
      Sd[o] = x;
      if (dfp && L.rowact[jrow]) emax = max(emax, (unsigned)df_exp_field(x));
    }
  } else if (dfp) {
    // value pairs (rows are even in length and 16-byte aligned): one 16-byte load per pair
    const int h2 = Nph / 2;
    for (int n = threadIdx.x; n < nact * h2; n += blockDim.x) {
      const int r = n / h2;
      const F64::C x = F64::ld16(saddr(buf) + 8u * (uint32_t)((int)L.arow[r] * ld + 2 * (n - r * h2)));
      emax = max(emax, max((unsigned)df_exp_field(x.re), (unsigned)df_exp_field(x.im)));
    }
  }
  int E = 0;
  if (dfp) {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (threadIdx.x == 0) L.misc[2] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&L.misc[2], (int)emax);
    __syncthreads();
    E = L.misc[2] - 1023;
    const uint32_t sb = saddr(buf);
    const int h2 = Nph / 2;
    for (int n = threadIdx.x; n < nact * h2; n += blockDim.x) {
      const int r = n / h2;
      const uint32_t a = sb + 8u * (uint32_t)((int)L.arow[r] * ld + 2 * (n - r * h2));
      const F64::C x = F64::ld16(a);
      P::st16(a, typename P::C{to_real<P>(x.re, E), to_real<P>(x.im, E)});
    }
  }
  __syncthreads();
  const int npairs = L.misc[0];
  const bool has_general = L.misc[1] != 0;
  const bool th_general = hyb && L.misc[4] != 0;

  ThetaAcc<P> TA;
  TA.S = saddr(buf);
  TA.ov = L.ov;
  TA.lin = L.lin;
  TA.g = L.g_th;
  TA.sel = L.thsel;
  TA.circ = L.circ;
  TA.hyb = hyb;
  TA.ld = ld;
  TA.Nth = Nth;
  TA.Nth8 = Nth & ~7;
  TA.h = Nph / 2;
  TA.M = 2 * Nth;
  TA.M8 = (2 * Nth) & ~7;
  TA.nseq = (Nph / 2 + 1) / 2;
  TA.lone_last = (Nph / 2) & 1;
  TA.odd = vi.parity != 0;
  TA.hodd = (Nph / 2) & 1;
  TA.b0 = 0;

  PhiAcc<P> PA;
  PA.S = saddr(buf);
  PA.ov = L.ov;
  PA.lin = L.lin;
  PA.pairs = L.pairs;
  PA.gtab = A.g_ph;
  PA.gbase = ((size_t)vi.cls * A.Nr + i) * (size_t)Nth * (Nph / 2 + 1);
  PA.gbase_alt = ((size_t)vi.alt_cls * A.Nr + i) * (size_t)Nth * (Nph / 2 + 1);
  PA.hyb = hyb;
  PA.ld = ld;
  PA.N = Nph;
  PA.N8 = Nph & ~7;
  PA.hN = Nph / 2;
  PA.hN8 = (Nph / 2) & ~7;
  PA.nh = Nph / 2 + 1;
  PA.b0 = 0;

  // the filter: theta pass then phi pass, or the reverse order for the transpose; the spectral form
  // runs both at once on shells with a theta pass
  if (SPEC && theta_on) {
    SpecAcc<P> SA;
    SA.S = saddr(buf);
    SA.lin = L.lin;
    SA.ld = ld;
    SA.N = Nth;
    SA.N8 = Nth & ~7;
    SA.b0 = 0;
    SA.parity = vi.parity;
    SA.nh = Nph / 2 + 1;
    SA.phi_first = io.transpose != 0;
    SA.gtab = A.g_ph;
    SA.gbase = PA.gbase;
    const int batch_sp = (int)(scratch_bytes(A) / (16 * (size_t)Nth));
    spectral_fn<P, LEN>(PA, SA, npairs, A.f_ph, A.f_sp, L.tw_ph, L.tw_th, L.g_th, K, A.batch_ph, batch_sp);
  } else
  for (int step = 0; step < 2; ++step) {
    if ((step == 0) != (io.transpose != 0)) {
      if (theta_on) {
        if (hyb) theta_pass_fn<P, LEN, false, true>(TA, A.f_th, L.tw_th, K, A.batch_th, th_general);
        else theta_pass_fn<P, LEN>(TA, A.f_th, L.tw_th, K, A.batch_th, false);
      }
    } else if (npairs) {
      if (hyb) phi_pass_fn<P, LEN, true>(PA, npairs, has_general, A.f_ph, L.tw_ph, K, A.batch_ph);
      else phi_pass_fn<P, LEN>(PA, npairs, has_general, A.f_ph, L.tw_ph, K, A.batch_ph);
    }
  }

  // store (streaming), with the output map; untransformed rows are still FP64
  const uint32_t sb = saddr(buf);
  if (in_place_sparse<LEN>(io)) {
    // in place: only the transformed rows change
    double2* dst = reinterpret_cast<double2*>(static_cast<double*>(io.out) + off);
    const int na = L.misc[3];
    for (int c = threadIdx.x; c < na * (Nph / 2); c += blockDim.x) {
      const int jrow = (int)L.arow[c / (Nph / 2)], k = 2 * (c % (Nph / 2));
      const int o = jrow * ld + k;
      const typename P::C v = P::ld16(sb + 8u * o);
      __stcs(dst + (jrow * Nph + k) / 2, make_double2(from_real<P>(v.re, E), from_real<P>(v.im, E)));
    }
    return;
  }
  if (!io.is_f32 && io.map_out == kOutNone) {
    // plain FP64 output: two values per 16-byte store (rows are even in length)
    double2* dst = reinterpret_cast<double2*>(static_cast<double*>(io.out) + off);
    const bool out16 = ((uintptr_t)dst & 15u) == 0;
    for (int n2 = threadIdx.x; n2 < npts / 2; n2 += blockDim.x) {
      const int n = 2 * n2, jrow = n / Nph;
      const int o = jrow * ld + n % Nph;
      double2 y;
      if (dfp && !L.rowact[jrow]) {
        const F64::C v = F64::ld16(sb + 8u * o);
        y = make_double2(v.re, v.im);
      } else {
        const typename P::C v = P::ld16(sb + 8u * o);
        y = make_double2(from_real<P>(v.re, E), from_real<P>(v.im, E));
      }
      if (out16) {
        __stcs(dst + n2, y);
      } else {
        __stcs(reinterpret_cast<double*>(dst) + n, y.x);
        __stcs(reinterpret_cast<double*>(dst) + n + 1, y.y);
      }
    }
    return;
  }
  for (int n = threadIdx.x; n < npts; n += blockDim.x) {
    const int jrow = n / Nph;
    const int o = jrow * ld + n % Nph;
    double y = (dfp && !L.rowact[jrow]) ? Sd[o] : from_real<P>(P::ld8(sb + 8u * o), E);
    if (io.map_out == kOutTanhGrad) {
      const double z = io.is_f32 ? (double)static_cast<const float*>(io.aux)[off + n]
                                 : static_cast<const double*>(io.aux)[off + n];
      y *= map_sech2<P>(z);
    }
    if (io.is_f32) __stcs(static_cast<float*>(io.out) + off + n, (float)y);
    else __stcs(static_cast<double*>(io.out) + off + n, y);
  }
}

template <class P, int LEN, bool HYB, bool SPEC = false>
__global__ void __launch_bounds__(512) shell_kernel(ShellArgs2 A, LaunchIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Layout<P> L = carve<P>(A, smem_raw);
  // a launch over a list of shells reads its shell index there (same encoding as the grid's)
  const int sidx = io.list ? __ldg(io.list + blockIdx.x) : (int)blockIdx.x;
  // the shell's copies first (bulk copies by warp 0, or cp.async by every thread; see
  // bulk_staging), then the twiddles (16-byte table entries copied as they are); the tables in
  // filter_shell are fetched while these are in flight. An in-place call copies only the rows a
  // pass transforms, once filter_shell knows them.
  const bool stage = !io.is_f32 && io.async_ok && !in_place_sparse<LEN>(io);
  const bool bulk = stage && bulk_staging<P>();
  if (bulk_staging<P>()) {
    if (threadIdx.x == 0) bar_init(L.bar);
    __syncthreads();  // the mbarrier is initialised
  }
  if (bulk && threadIdx.x < 32) issue_shell_copies<LEN>(A, io, sidx, L.buf, L.bar);
  if (stage && !bulk) issue_shell_async<LEN>(A, io, sidx, L.buf);
  const typename P::C* twth_g = static_cast<const typename P::C*>(A.tw_th);
  const typename P::C* twph_g = static_cast<const typename P::C*>(A.tw_ph);
  for (int n = threadIdx.x; n < 2 * A.Nth; n += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(L.tw_th + 16u * n), "l"(twth_g + n) : "memory");
  for (int n = threadIdx.x; n < A.Nph; n += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(L.tw_ph + 16u * n), "l"(twph_g + n) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  Consts<P> K;
  K.c8 = P::from_tab(A.consts, 0);
  K.s3 = P::from_tab(A.consts, 1);

  filter_shell<P, LEN, HYB, SPEC>(A, io, L, L.buf, sidx, K, bulk);
}


// ------------------------------------------------------------------ sparse shells: ring-pair units

// A shell whose theta pass is the identity (exponential or sharp filter, l_max >= Ntheta) changes
// only in its active phi rings. The units kernel filters the active ring pairs of many such shells:
// a CTA stages kUnits pairs (rows 2u and 2u + 1 of a small row buffer, u < kUnits), each with its
// own power-of-two scale, and runs the phi pass on them with the shell kernel's stages; the copy
// kernel moves the shells' other rows (out-of-place calls). Several such CTAs fit an SM, where a
// whole-shell CTA would run a few pairs with most of its threads idle.
constexpr int kUnits = 8;
constexpr int kUnitThreads = 256;

// PhiAcc over the row buffer: the pair list is (2u | general << 30, 2u + 1), and row_tab[r] is the
// element offset of row r's multipliers in the global table. A lone middle ring (Ntheta odd) is
// paired with a zero row that takes its multipliers (its output is zero and is not stored).
template <class P>
struct PhiUnitsAcc : PhiAcc<P> {
  using T = typename P::T;
  using Seq = typename PhiAcc<P>::Seq;
  const unsigned* row_tab;
  __device__ __forceinline__ T row_mult(int r, int m) const {
    return P::from_tab(this->gtab, (size_t)row_tab[r] + (m <= this->hN ? m : this->N - m));
  }
  __device__ __forceinline__ T mult(const Seq& s, int m) const { return row_mult(s.j1, m); }
  __device__ __forceinline__ void mult2(const Seq& s, int m, T& f1, T& f2) const {
    f1 = row_mult(s.j1, m);
    f2 = row_mult(s.j2, m);
  }
};

__host__ __device__ __forceinline__ size_t units_smem(const ShellArgs2& a) {
  auto up = [](size_t x) { return (x + 15) / 16 * 16; };
  size_t s = up(8 * (size_t)(2 * kUnits) * a.ldS);  // rows
  s += up(16 * (size_t)kUnits * a.Nph);              // FFT scratch
  s += up(16 * (size_t)a.Nph);                       // twiddles
  s += up(sizeof(int2) * kUnits);                    // pair list
  s += up(sizeof(unsigned) * 2 * kUnits);            // row_tab
  s += up(sizeof(int) * (kUnits + 4));               // per-unit exponents, flags
  return s;
}

template <class P, int LEN>
__global__ void __launch_bounds__(kUnitThreads) units_kernel(ShellArgs2 A, LaunchIO io, const int* units, int nunits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool dfp = std::is_same<P, DF>::value;
  const int Nth = LEN ? LEN / 2 : A.Nth, Nph = LEN ? LEN : A.Nph, ld = LEN ? LEN + 2 : A.ldS;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = smem_raw + off;
    off = (off + bytes + 15) / 16 * 16;
    return p;
  };
  unsigned char* rows = take(8 * (size_t)(2 * kUnits) * ld);
  const uint32_t S = saddr(rows);
  const uint32_t lin = saddr(take(16 * (size_t)kUnits * Nph));
  const uint32_t tw = saddr(take(16 * (size_t)Nph));
  int2* pairs = reinterpret_cast<int2*>(take(sizeof(int2) * kUnits));
  unsigned* row_tab = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * 2 * kUnits));
  int* ue = reinterpret_cast<int*>(take(sizeof(int) * (kUnits + 4)));  // [u] exponent, [kUnits] general
  const int u0 = blockIdx.x * kUnits, nu = min(kUnits, nunits - u0);
  const int h2 = Nph / 2;

  // the pairs' rows (16-byte pieces), then the twiddles
  for (int c = threadIdx.x; c < nu * 2 * h2; c += blockDim.x) {
    const int r = c / h2, k2 = c - r * h2, u = r >> 1;
    const int e = units[u0 + u], j = e % Nth, sh = e / Nth;  // sh = v * Nr + i
    const int row = (r & 1) ? Nth - 1 - j : j;
    if ((r & 1) && row == j) {  // lone middle ring: a zero partner row
      F64::st16(S + (uint32_t)(r * ld + 2 * k2) * 8u, F64::C{0.0, 0.0});
      continue;
    }
    const double* src = static_cast<const double*>(io.in) + ((size_t)sh * Nth + row) * Nph + 2 * k2;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(S + (uint32_t)(r * ld + 2 * k2) * 8u), "l"(src)
                 : "memory");
  }
  const typename P::C* twph_g = static_cast<const typename P::C*>(A.tw_ph);
  for (int n = threadIdx.x; n < Nph; n += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tw + 16u * n), "l"(twph_g + n) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (threadIdx.x == 0) ue[kUnits] = 0;
  __syncthreads();
  if (threadIdx.x < nu) {
    const int u = threadIdx.x;
    const int e = units[u0 + u], j = e % Nth, sh = e / Nth, v = sh / A.Nr, i = sh - v * A.Nr, jj = Nth - 1 - j;
    const int cls = A.var[v].cls;
    const uint8_t* ri = A.ring_info + ((size_t)cls * A.Nr + i) * Nth;
    const int g = jj != j ? (ri[j] >> 1) & 1 : 0;  // bit 1: the two rings' multipliers differ
    pairs[u] = make_int2(2 * u | (g << 30), 2 * u + 1);
    const unsigned base = (unsigned)(((size_t)cls * A.Nr + i) * (size_t)Nth) * (unsigned)(Nph / 2 + 1);
    row_tab[2 * u] = base + (unsigned)j * (Nph / 2 + 1);
    row_tab[2 * u + 1] = base + (unsigned)jj * (Nph / 2 + 1);  // jj == j for a lone ring
    if (g) atomicOr(&ue[kUnits], 1);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // compensated FP32: one scale per unit (its rows' largest exponent), conversion in place
  if constexpr (dfp) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int u = warp; u < nu; u += blockDim.x >> 5) {
      const int nr = 2;
      unsigned em = 0;
      for (int c = lane; c < nr * h2; c += 32) {
        const int r = 2 * u + c / h2;
        const F64::C x = F64::ld16(S + 8u * (uint32_t)(r * ld + 2 * (c % h2)));
        em = max(em, max((unsigned)df_exp_field(x.re), (unsigned)df_exp_field(x.im)));
      }
      em = __reduce_max_sync(0xffffffffu, em);
      const int E = (int)em - 1023;
      if (lane == 0) ue[u] = E;
      for (int c = lane; c < nr * h2; c += 32) {
        const int r = 2 * u + c / h2;
        const uint32_t a = S + 8u * (uint32_t)(r * ld + 2 * (c % h2));
        const F64::C x = F64::ld16(a);
        P::st16(a, typename P::C{to_real<P>(x.re, E), to_real<P>(x.im, E)});
      }
    }
    __syncthreads();
  }
  Consts<P> K;
  K.c8 = P::from_tab(A.consts, 0);
  K.s3 = P::from_tab(A.consts, 1);
  PhiUnitsAcc<P> PA;
  PA.S = S;
  PA.ov = 0;
  PA.lin = lin;
  PA.pairs = pairs;
  PA.gtab = A.g_ph;
  PA.gbase = 0;
  PA.gbase_alt = 0;
  PA.hyb = false;
  PA.ld = ld;
  PA.N = Nph;
  PA.N8 = Nph & ~7;
  PA.hN = Nph / 2;
  PA.hN8 = (Nph / 2) & ~7;
  PA.nh = Nph / 2 + 1;
  PA.b0 = 0;
  PA.row_tab = row_tab;
  PA.template fix<LEN>();
  run_pass<P, PhiUnitsAcc<P>, LEN>(PA, Nph, nu, A.f_ph, tw, K, ue[kUnits] != 0);
  // store the filtered rows (the last stage synchronised the block)
  for (int c = threadIdx.x; c < nu * 2 * h2; c += blockDim.x) {
    const int r = c / h2, k2 = c - r * h2, u = r >> 1;
    const int e = units[u0 + u], j = e % Nth, sh = e / Nth;
    const int row = (r & 1) ? Nth - 1 - j : j;
    if ((r & 1) && row == j) continue;  // the zero partner of a lone ring
    const int E = dfp ? ue[u] : 0;
    const typename P::C y = P::ld16(S + 8u * (uint32_t)(r * ld + 2 * k2));
    double2* dst = reinterpret_cast<double2*>(static_cast<double*>(io.out) + ((size_t)sh * Nth + row) * Nph) + k2;
    __stcs(dst, make_double2(from_real<P>(y.re, E), from_real<P>(y.im, E)));
  }
}

template <class P, int LEN>
cudaError_t launch_units_impl(const ShellArgs2& a, size_t smem, const LaunchIO& io, const int* units, int nunits,
                              cudaStream_t s) {
  const dim3 grid((unsigned)((nunits + kUnits - 1) / kUnits));
  units_kernel<P, LEN><<<grid, kUnitThreads, smem, s>>>(a, io, units, nunits);
  return cudaGetLastError();
}

template <class P, int LEN>
cudaError_t set_attr_units_impl(int bytes) {
  return cudaFuncSetAttribute(units_kernel<P, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ------------------------------------------------------------------ cluster-pair kernel (large shells)

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ uint4 ld_peer16(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ double ld_peer8(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}

// The detector's view of one CTA of a pair (hybrid fields): its buffer A holds every row of the
// global meridian blocks r and r + 2 (Nphi/4 columns each) at local columns [0, Nphi/4) and
// [Nphi/4, Nphi/2), so local column c and c + Nphi/4 are the two meridians of a circle. A ring's
// cells next to a block edge have their phi neighbour in the peer's buffer (same layout), read
// through distributed shared memory.
template <int LEN>
struct DetHalf {
  static constexpr bool kPair = true;
  uint32_t S;
  int nth, nph, ld, r;
  __device__ __forceinline__ int Nth() const { return LEN ? LEN / 2 : nth; }
  __device__ __forceinline__ int W() const { return LEN ? LEN / 2 : nph / 2; }
  __device__ __forceinline__ int lds() const { return LEN ? LEN / 2 + 2 : ld; }
  __device__ __forceinline__ double at(int j, int c) const { return F64::ld8(S + 8u * (uint32_t)(j * lds() + c)); }
  __device__ __forceinline__ double nbr(int j, int c, int dir) const {
    const int QB = W() / 2, Nph = 2 * W();
    int g = (c < QB ? r * QB + c : (r + 2) * QB + (c - QB)) + dir;  // global column of the neighbour
    g = g < 0 ? Nph - 1 : (g == Nph ? 0 : g);
    const int blk = g / QB;
    const uint32_t a = S + 8u * (uint32_t)(j * lds() + (g - blk * QB) + (blk >= 2 ? QB : 0));
    return (blk & 1) == r ? F64::ld8(a) : ld_peer8(peer_addr(a, 1 - r));
  }
  __device__ __forceinline__ void pair_sync() const { cluster_sync(); }
  __device__ __forceinline__ int peer_int(const int* p) const {
    unsigned v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(peer_addr(saddr(p), 1 - r)));
    return (int)v;
  }
  __device__ __forceinline__ int peer_u8(const unsigned char* p) const {
    unsigned v;
    asm volatile("ld.shared::cluster.u8 %0, [%1];" : "=r"(v) : "r"(peer_addr(saddr(p), 1 - r)));
    return (int)v;
  }
};

__device__ __forceinline__ void st_local16(uint32_t a, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

template <class P>
struct LayoutCl {
  uint32_t A, B, lin, ov, tw_th, tw_ph, g_th;
  int2* pairs;
  int* misc;               // [0] pair count, [1] general flag, [2] exponent; hybrid fields: [4] mixed
                           // circle pairs, [5] some circle fired (over the pair), [6], [7] scratch
  uint32_t rowact;         // shared address of the row flags: a pass transforms row j (1) or not (0)
  unsigned char* circ;     // hybrid fields: detector flags of this CTA's theta circles [Nphi/4],
  unsigned char* ring;     //   of the phi rings [Ntheta] (over the pair),
  unsigned char* thsel;    //   and the table choice of this CTA's theta sequences [(Nphi/4 + 1)/2]
};

// Shared memory of one CTA of a pair: A (all rows, half the columns), B (half of the rows, the other
// half of the columns), tables. The FFT scratch of the theta pass is B (not yet filled, or already
// read by the peer); that of the phi pass is the peer's rows of A (not yet filled, or already read).
__host__ __device__ __forceinline__ size_t cl_ld(const ShellArgs2& A) { return (size_t)A.Nph / 2 + 2; }

template <class P>
__device__ LayoutCl<P> carve_cl(const ShellArgs2& A, unsigned char* base) {
  LayoutCl<P> L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off = (off + bytes + 15) / 16 * 16;
    return p;
  };
  L.A = saddr(take(8 * (size_t)A.Nth * cl_ld(A)));
  L.B = saddr(take(8 * (size_t)(A.Nth / 2) * cl_ld(A)));
  L.lin = 0;
  L.ov = saddr(take(16 * (size_t)max(2 * A.Nth, A.Nph)));
  L.tw_th = saddr(take(16 * 2 * (size_t)A.Nth));
  L.tw_ph = saddr(take(16 * (size_t)A.Nph));
  L.g_th = saddr(take(16 * (size_t)(A.Nth + 1)));  // two rows: a hybrid field's Gaussian one second
  L.pairs = reinterpret_cast<int2*>(take(sizeof(int2) * (size_t)(A.Nth / 2 + 1)));
  L.misc = reinterpret_cast<int*>(take(sizeof(int) * 8));
  L.rowact = saddr(take((size_t)A.Nth));
  L.circ = take((size_t)(A.Nph / 4 + A.Nth + (A.Nph / 4 + 1) / 2));
  L.ring = L.circ + A.Nph / 4;
  L.thsel = L.ring + A.Nth;
  return L;
}

__device__ __forceinline__ bool row_on(uint32_t flags, int j) {
  unsigned v;
  asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(flags + (uint32_t)j));
  return v != 0;
}

template <class P>
size_t shell_smem_cl(const ShellArgs2& a) {
  auto up = [](size_t x) { return (x + 15) / 16 * 16; };
  size_t s = up(8 * (size_t)a.Nth * cl_ld(a));
  s += up(8 * (size_t)(a.Nth / 2) * cl_ld(a));
  s += up(16 * (size_t)std::max(2 * a.Nth, a.Nph));
  s += up(16 * 2 * (size_t)a.Nth);
  s += up(16 * (size_t)a.Nph);
  s += up(16 * (size_t)(a.Nth + 1));
  s += up(sizeof(int2) * (size_t)(a.Nth / 2 + 1));
  s += up(sizeof(int) * 8);
  s += up((size_t)a.Nth);
  s += up((size_t)(a.Nph / 4 + a.Nth + (a.Nph / 4 + 1) / 2));
  return s;
}

// Global column c of a shell row -> (is it in this rank's blocks {r, r+2}, local column).
__device__ __forceinline__ bool cl_mine(int c, int QB, int r, int* lc) {
  const int blk = c / QB;
  *lc = (c - blk * QB) + (blk >= 2 ? QB : 0);
  return blk == r || blk == 2 + r;
}
__device__ __forceinline__ int cl_brow(int j, int Nth, int r) {
  const int q = Nth / 4;
  return j < Nth / 2 ? j - q * r : q + (j - (Nth - (r + 1) * q));
}
__device__ __forceinline__ bool cl_own_row(int j, int Nth, int r) {
  const int q = Nth / 4;
  return (j >= q * r && j < q * (r + 1)) || (j >= Nth - (r + 1) * q && j < Nth - r * q);
}

// One shell per cluster pair; Ntheta % 4 == 0, Nphi % 8 == 0. HYB: the variant for launches with
// hybrid fields (forward order only).
template <class P, int LEN, bool HYB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512) shell_kernel_cl(ShellArgs2 A, LaunchIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool dfp = std::is_same<P, DF>::value;
  const LayoutCl<P> L = carve_cl<P>(A, smem_raw);
  const int r = (int)cluster_rank();
  const int sidx = blockIdx.x / 2;
  int v, i;
  const size_t off = shell_offset(A, io, sidx, &v, &i);
  const VarInfo vi = A.var[v];
  // compile-time sizes for the fixed lengths
  const int Nth = LEN ? LEN / 2 : A.Nth, Nph = LEN ? LEN : A.Nph, QB = Nph / 4;
  const int ldc = LEN ? LEN / 2 + 2 : (int)cl_ld(A);
  const bool fwd = io.transpose == 0;
  const bool hyb = HYB && fwd && vi.kind == SPH_FILTER_HYBRID;  // the same on both CTAs of the pair

  for (int n = threadIdx.x; n < 2 * Nth; n += blockDim.x)
    P::st16(L.tw_th + 16u * n, static_cast<const typename P::C*>(A.tw_th)[n]);
  for (int n = threadIdx.x; n < Nph; n += blockDim.x)
    P::st16(L.tw_ph + 16u * n, static_cast<const typename P::C*>(A.tw_ph)[n]);
  Consts<P> K;
  K.c8 = P::from_tab(A.consts, 0);
  K.s3 = P::from_tab(A.consts, 1);

  // load: forward order takes every row of blocks {r, r+2} into A; the transpose order takes this
  // rank's rows, blocks {r, r+2} into A and the others into B. Raw FP64 first (cp.async, 16-byte
  // pieces, when the input is FP64 and 16-byte aligned).
  const double* srcd = static_cast<const double*>(io.in) + off;
  const float* srcf = static_cast<const float*>(io.in) + off;
  const int rows = fwd ? Nth : Nth / 2;
  auto row_of = [&](int jr) {
    return fwd ? jr : (jr < Nth / 4 ? r * (Nth / 4) + jr : Nth - (r + 1) * (Nth / 4) + (jr - Nth / 4));
  };
  auto addr_of = [&](int j, int c) {
    int lc;
    const bool mine = cl_mine(c, QB, r, &lc);
    return mine ? L.A + (uint32_t)(j * ldc + lc) * 8u : L.B + (uint32_t)(cl_brow(j, Nth, r) * ldc + lc) * 8u;
  };
  const int cols = fwd ? Nph / 2 : Nph;  // columns loaded per row
  auto col_of = [&](int cc) {            // cc-th loaded column of a row
    if (!fwd) return cc;
    return cc < QB ? r * QB + cc : (2 + r) * QB + (cc - QB);
  };
  if (!io.is_f32 && io.async_ok) {
    for (int e = threadIdx.x; e < rows * (cols / 2); e += blockDim.x) {
      const int jr = e / (cols / 2), c = col_of(2 * (e - jr * (cols / 2)));
      const int j = row_of(jr);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(addr_of(j, c)), "l"(srcd + (size_t)j * Nph + c)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int jr = e / cols, c = col_of(e - jr * cols);
      const int j = row_of(jr);
      const double x = io.is_f32 ? (double)__ldcs(srcf + (size_t)j * Nph + c) : __ldcs(srcd + (size_t)j * Nph + c);
      F64::st8(addr_of(j, c), x);
    }
    __syncthreads();
  }
  if (hyb) {
    // Jameson's detector on the raw FP64 values; ring flags and "a circle fired" come out combined
    // over the pair, so both CTAs take the same rows and the same theta decision
    DetHalf<LEN> geo;
    geo.S = L.A;
    geo.nth = Nth;
    geo.nph = Nph;
    geo.ld = ldc;
    geo.r = r;
    detect_shell(geo, vi.parity != 0, A.eps, A.eps_m, A.eps_p, L.circ, L.ring, L.misc);
    __syncthreads();
  }
  // rows a pass transforms: every row when the theta pass runs, else the rows of active ring pairs
  // (the same rows on both ranks); only these are converted to pairs, the rest stay FP64
  {
    const bool th_on = vi.kind == SPH_FILTER_GAUSS || A.lmax[vi.cls * A.Nr + i] < (double)Nth || (hyb && L.misc[5] != 0);
    const uint8_t* ri = A.ring_info + ((size_t)vi.cls * A.Nr + i) * Nth;
    for (int j = threadIdx.x; j < Nth; j += blockDim.x) {
      const bool fire = hyb && (L.ring[j] || L.ring[Nth - 1 - j]);
      asm volatile("st.shared.u8 [%0], %1;" ::"r"(L.rowact + (uint32_t)j),
                   "r"((th_on || fire || ((ri[j] | ri[Nth - 1 - j]) & 1)) ? 1u : 0u));
    }
  }
  __syncthreads();
  unsigned emax = 0;
  if (io.map_in == kMapTanh || dfp) {
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int jr = e / cols, c = col_of(e - jr * cols);
      const int j = row_of(jr);
      const uint32_t a = addr_of(j, c);
      double x = F64::ld8(a);
      if (io.map_in == kMapTanh) {
        x = map_tanh<P>(x);
        F64::st8(a, x);
      }
      if (dfp && row_on(L.rowact, j)) emax = max(emax, (unsigned)df_exp_field(x));
    }
  }
  int E = 0;
  if (dfp) {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (threadIdx.x == 0) L.misc[2] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&L.misc[2], (int)emax);
    cluster_sync();  // both halves' maxima are in place
    const uint32_t mine = saddr(&L.misc[2]);
    unsigned other;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(other) : "r"(peer_addr(mine, 1 - r)));
    E = max(L.misc[2], (int)other) - 1023;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int jr = e / cols, c = col_of(e - jr * cols);
      const int j = row_of(jr);
      if (!row_on(L.rowact, j)) continue;
      const uint32_t a = addr_of(j, c);
      P::st8(a, to_real<P>(F64::ld8(a), E));
    }
  }

  // per-shell tables (a hybrid field's Gaussian theta row after its exponential one)
  const double lmax = A.lmax[vi.cls * A.Nr + i];
  const bool theta_on = vi.kind == SPH_FILTER_GAUSS || lmax < (double)Nth || (hyb && L.misc[5] != 0);
  const uint8_t* ring_info = A.ring_info + ((size_t)vi.cls * A.Nr + i) * Nth;
  const uint8_t* ring_alt = A.ring_info + ((size_t)vi.alt_cls * A.Nr + i) * Nth;
  const size_t gth_base = ((size_t)vi.cls * A.Nr + i) * (Nth + 1);
  const size_t gth_alt = ((size_t)vi.alt_cls * A.Nr + i) * (Nth + 1);
  for (int n = threadIdx.x; n < (hyb ? 2 : 1) * (Nth + 1); n += blockDim.x)
    P::st8(L.g_th + 8u * n, P::from_tab(A.g_th, n <= Nth ? gth_base + n : gth_alt + (n - (Nth + 1))));
  if (threadIdx.x == 0) {
    int np = 0, gen = 0;
    const int q = Nth / 4;
    for (int j = q * r; j < q * (r + 1); ++j) {
      const int jj = Nth - 1 - j;
      const uint8_t a = ring_info[j], b = ring_info[jj];
      // hybrid field: a ring whose detector fired takes the Gaussian table (never the identity)
      const int fa = hyb ? L.ring[j] : 0, fb = hyb ? L.ring[jj] : 0;
      if (!((a | b) & 1) && !fa && !fb) continue;
      const int g = fa != fb ? 1 : ((fa ? ring_alt[j] : a) >> 1) & 1;
      gen |= g;
      L.pairs[np++] = make_int2(j | (g << 30) | (fa << 29) | (fb << 28), jj);
    }
    L.misc[0] = np;
    L.misc[1] = gen;
  }
  if (hyb && threadIdx.x >= 32 && threadIdx.x < 64) {
    // table of each of this CTA's theta sequences (circles 2b, 2b+1): 0 exponential, 1 Gaussian,
    // 2 one of each (split multiply); a lone last circle counts twice
    const int lane = threadIdx.x - 32, hc = Nph / 4, nseq = (hc + 1) / 2;
    int gth = 0;
    for (int b0 = 0; b0 < nseq; b0 += 32) {
      const int b = b0 + lane;
      int t = 0;
      if (b < nseq) {
        const int c1 = L.circ[2 * b], c2 = 2 * b + 1 < hc ? L.circ[2 * b + 1] : c1;
        t = c1 == c2 ? c1 : 2;
        L.thsel[b] = (unsigned char)t;
      }
      gth |= __any_sync(0xffffffffu, t == 2) ? 1 : 0;
    }
    if (lane == 0) L.misc[4] = gth;
  }
  __syncthreads();
  const int npairs = L.misc[0];
  const bool has_general = L.misc[1] != 0;
  const bool th_general = hyb && L.misc[4] != 0;

  ThetaAcc<P> TA;
  TA.S = L.A;
  TA.ov = L.ov;
  TA.lin = L.B;
  TA.g = L.g_th;
  TA.ld = ldc;
  TA.Nth = Nth;
  TA.Nth8 = Nth & ~7;
  TA.h = Nph / 4;
  TA.M = 2 * Nth;
  TA.M8 = (2 * Nth) & ~7;
  TA.nseq = (Nph / 4 + 1) / 2;
  TA.lone_last = (Nph / 4) & 1;
  TA.odd = vi.parity != 0;
  TA.hodd = (Nph / 4) & 1;
  TA.b0 = 0;
  TA.sel = L.thsel;
  TA.circ = L.circ;
  TA.hyb = hyb;

  PhiSplitAcc<P> PA;
  PA.A = L.A;
  PA.Bm = L.B;
  {
    const int q = Nth / 4, ro = 1 - r;
    PA.lin0 = L.A + (uint32_t)(q * ro * ldc) * 8u;
    PA.lin1 = L.A + (uint32_t)((Nth - (ro + 1) * q) * ldc) * 8u;
    PA.cap = (q * ldc * 8) / (16 * Nph);
  }
  PA.pairs = L.pairs;
  PA.gtab = A.g_ph;
  PA.gbase = ((size_t)vi.cls * A.Nr + i) * (size_t)Nth * (Nph / 2 + 1);
  PA.gbase_alt = ((size_t)vi.alt_cls * A.Nr + i) * (size_t)Nth * (Nph / 2 + 1);
  PA.hyb = hyb;
  PA.ld = ldc;
  PA.N = Nph;
  PA.N8 = Nph & ~7;
  PA.QB = QB;
  PA.QB8 = QB & ~7;
  PA.Nth = Nth;
  PA.r = r;
  PA.hN = Nph / 2;
  PA.nh = Nph / 2 + 1;
  PA.b0 = 0;

  // exchange through the peer's shared memory: forward, this rank's rows of the peer's blocks (the
  // peer's A -> our B); transpose, the peer's rows of our blocks (the peer's B -> our A)
  auto exchange = [&]() {
    cluster_sync();  // the peer's first pass is complete
    const int half = Nph / 2;  // local columns of a row
    const int q = Nth / 4;
    for (int e = threadIdx.x; e < (Nth / 2) * (half / 2); e += blockDim.x) {
      const int jr = e / (half / 2), c2 = 2 * (e - jr * (half / 2));
      if (fwd) {
        const int j = jr < q ? r * q + jr : Nth - (r + 1) * q + (jr - q);
        const uint4 val = ld_peer16(peer_addr(L.A + (uint32_t)(j * ldc + c2) * 8u, 1 - r));
        st_local16(L.B + (uint32_t)(cl_brow(j, Nth, r) * ldc + c2) * 8u, val);
      } else {
        const int ro = 1 - r;
        const int j = jr < q ? ro * q + jr : Nth - (ro + 1) * q + (jr - q);
        const uint4 val = ld_peer16(peer_addr(L.B + (uint32_t)(cl_brow(j, Nth, ro) * ldc + c2) * 8u, ro));
        st_local16(L.A + (uint32_t)(j * ldc + c2) * 8u, val);
      }
    }
    cluster_sync();  // both reads are done before either side writes the rows the peer read
  };

  if (fwd) {
    if (theta_on) {
      if (hyb) theta_pass_fn<P, LEN, true, true>(TA, A.f_th, L.tw_th, K, A.batch_th, th_general);
      else theta_pass_fn<P, LEN, true>(TA, A.f_th, L.tw_th, K, A.batch_th, false);
    }
    exchange();
    if (npairs) {
      if (hyb) phi_split_pass_fn<P, LEN, true>(PA, npairs, has_general, A.f_ph, L.tw_ph, K, A.batch_ph);
      else phi_split_pass_fn<P, LEN>(PA, npairs, has_general, A.f_ph, L.tw_ph, K, A.batch_ph);
    }
  } else {
    if (npairs) phi_split_pass_fn<P, LEN>(PA, npairs, has_general, A.f_ph, L.tw_ph, K, A.batch_ph);
    exchange();
    if (theta_on) theta_pass_fn<P, LEN, true>(TA, A.f_th, L.tw_th, K, A.batch_th, false);
  }
  __syncthreads();

  // store: forward, this rank's rows (A and B); transpose, every row of blocks {r, r+2} (A)
  const int store_rows = fwd ? Nth / 2 : Nth;
  for (int e = threadIdx.x; e < store_rows * Nph; e += blockDim.x) {
    const int jr = e / Nph, c = e - jr * Nph;
    int j = jr;
    if (fwd) j = jr < Nth / 4 ? r * (Nth / 4) + jr : Nth - (r + 1) * (Nth / 4) + (jr - Nth / 4);
    int lc;
    const bool mine = cl_mine(c, QB, r, &lc);
    if (!fwd && !mine) continue;
    const uint32_t a = mine ? L.A + (uint32_t)(j * ldc + lc) * 8u : L.B + (uint32_t)(cl_brow(j, Nth, r) * ldc + lc) * 8u;
    double y = (dfp && !row_on(L.rowact, j)) ? F64::ld8(a) : from_real<P>(P::ld8(a), E);
    const size_t o = off + (size_t)j * Nph + c;
    if (io.map_out == kOutTanhGrad) {
      const double z = io.is_f32 ? (double)static_cast<const float*>(io.aux)[o] : static_cast<const double*>(io.aux)[o];
      y *= map_sech2<P>(z);
    }
    if (io.is_f32) __stcs(static_cast<float*>(io.out) + o, (float)y);
    else __stcs(static_cast<double*>(io.out) + o, y);
  }
}

template <class P, int LEN, bool HYB>
cudaError_t launch_cl_impl(const ShellArgs2& a, int threads, size_t smem, const LaunchIO& io, cudaStream_t s) {
  const dim3 grid((unsigned)(2 * io.var_count * a.Nr));
  shell_kernel_cl<P, LEN, HYB><<<grid, threads, smem, s>>>(a, io);
  return cudaGetLastError();
}

template <class P, int LEN, bool HYB>
cudaError_t set_attr_cl_impl(int bytes) {
  return cudaFuncSetAttribute(shell_kernel_cl<P, LEN, HYB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class P>
size_t shell_smem(const ShellArgs2& a) {
  auto up = [](size_t x) { return (x + 15) / 16 * 16; };
  size_t s = up(8 * (size_t)a.Nth * a.ldS);
  s += up(scratch_bytes(a));
  s += up(16 * (size_t)std::max(2 * a.Nth, a.Nph));
  s += up(16 * 2 * (size_t)a.Nth);
  s += up(16 * (size_t)a.Nph);
  s += up(16 * (size_t)(a.Nth + 1));
  s += up(sizeof(int2) * (size_t)(a.Nth / 2 + 1));
  s += up(sizeof(int) * 8);
  s += up((size_t)a.Nth);
  s += up(sizeof(unsigned short) * (size_t)a.Nth);
  s += up((size_t)(a.Nph / 2 + a.Nth + (a.Nph / 2 + 1) / 2));
  s += 16;  // mbarrier and the wait's outcome
  return s;
}

template <class P, int LEN, bool HYB, bool SPEC = false>
cudaError_t launch_impl(const ShellArgs2& a, int threads, size_t smem, const LaunchIO& io, cudaStream_t s) {
  const dim3 grid((unsigned)(io.list ? io.nlist : io.var_count * a.Nr));
  shell_kernel<P, LEN, HYB, SPEC><<<grid, threads, smem, s>>>(a, io);
  return cudaGetLastError();
}

template <class P, int LEN, bool HYB, bool SPEC = false>
cudaError_t set_attr_impl(int bytes) {
  return cudaFuncSetAttribute(shell_kernel<P, LEN, HYB, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class P>
size_t smem_impl(const ShellArgs2& a) {
  return shell_smem<P>(a);
}

}  // namespace shellk
}  // namespace sph
