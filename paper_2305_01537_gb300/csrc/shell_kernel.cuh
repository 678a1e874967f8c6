// Shell kernel of the double FFT filter (arXiv:2305.01537, Sec. II.C), register-staged in-place form.
// Included by shell_inst.cu, which the build compiles once per (precision, FFT length) pair.
//
// One CTA filters one (field, shell) pair. The shell (Ntheta x Nphi values) is staged once in
// shared memory, which is also the only FFT buffer: every FFT stage loads all of its butterflies'
// inputs into registers, synchronises, and stores the outputs back into the same memory. All
// sequences of a pass are transformed in one batch, so each stage holds the whole shell in
// registers (at most 16 complex values per thread).
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
//
// The arithmetic policy is FP64 (F64) or compensated FP32 pairs (DF, about 48-bit significands,
// with a per-shell power-of-two scale). Multipliers f(|l|)/N and twiddles come from FP64 tables
// built on the host.
#pragma once

#include <type_traits>

#include "df32.h"
#include "internal.h"

namespace sph {
namespace shellk {


// ------------------------------------------------------------------ arithmetic policies

struct F64 {
  using T = double;
  using Store = double;
  struct C {
    double re, im;
  };
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T half(T a) { return 0.5 * a; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T ld(const Store* p) { return *p; }
  static __device__ __forceinline__ void st(Store* p, T v) { *p = v; }
  static __device__ __forceinline__ T from_tab(const void* tab, size_t i) {
    return __ldg(static_cast<const double*>(tab) + i);
  }
  static __device__ __forceinline__ C ld_tw(const void* tab, int i) {
    const double2 w = static_cast<const double2*>(tab)[i];
    return C{w.x, w.y};
  }
  static __device__ __forceinline__ C cmul(C a, C w) {
    return C{fma(a.re, w.re, -a.im * w.im), fma(a.re, w.im, a.im * w.re)};
  }
};

struct DF {
  using T = df;
  using Store = float2;
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
  static __device__ __forceinline__ df mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return df{h, __fsub_rn(e, __fsub_rn(h, p))};
  }
  static __device__ __forceinline__ df half(df a) { return df{0.5f * a.hi, 0.5f * a.lo}; }
  static __device__ __forceinline__ df zero() { return df{0.0f, 0.0f}; }
  static __device__ __forceinline__ df ld(const Store* p) {
    const float2 v = *p;
    return df{v.x, v.y};
  }
  static __device__ __forceinline__ void st(Store* p, df v) { *p = make_float2(v.hi, v.lo); }
  static __device__ __forceinline__ df from_tab(const void* tab, size_t i) {
    const float2 v = __ldg(static_cast<const float2*>(tab) + i);
    return df{v.x, v.y};
  }
  static __device__ __forceinline__ C ld_tw(const void* tab, int i) {
    const float4 w = static_cast<const float4*>(tab)[i];
    return C{df{w.x, w.y}, df{w.z, w.w}};
  }
  // a.hi*b.hi - c.hi*d.hi + (low-order terms), renormalised: one part of a complex product.
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
    const float h = __fadd_rn(s, t);
    return df{h, __fsub_rn(t, __fsub_rn(h, s))};
  }
  static __device__ __forceinline__ C cmul(C a, C w) {
    return C{dot2(a.re, w.re, a.im, w.im), dot2(a.re, w.im, neg(a.im), w.re)};
  }
};

template <class P>
struct Cx {
  using C = typename P::C;
  using T = typename P::T;
  static __device__ __forceinline__ C add(C a, C b) { return C{P::add(a.re, b.re), P::add(a.im, b.im)}; }
  static __device__ __forceinline__ C sub(C a, C b) { return C{P::sub(a.re, b.re), P::sub(a.im, b.im)}; }
  static __device__ __forceinline__ C scale(C a, T g) { return C{P::mul(a.re, g), P::mul(a.im, g)}; }
  static __device__ __forceinline__ C neg(C a) { return C{P::neg(a.re), P::neg(a.im)}; }
  // multiply by DIR * i
  template <int DIR>
  static __device__ __forceinline__ C mul_i(C v) {
    return DIR < 0 ? C{v.im, P::neg(v.re)} : C{P::neg(v.im), v.re};
  }
  static __device__ __forceinline__ C conj_tw(C w) { return C{w.re, P::neg(w.im)}; }
};

// Constants the radix kernels need, in the policy's precision (filled from FP64 host values).
template <class P>
struct Consts {
  typename P::T c8;   // sqrt(1/2)
  typename P::T s3;   // sqrt(3)/2
};

// ------------------------------------------------------------------ in-register DFTs

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
    const typename P::C m{P::sub(v[0].re, P::half(t.re)), P::sub(v[0].im, P::half(t.im))};
    const auto w = X::template mul_i<DIR>(X::scale(s, k.s3));
    v[0] = X::add(v[0], t);
    v[1] = X::add(m, w);
    v[2] = X::sub(m, w);
  }
};

// ------------------------------------------------------------------ pass accessors

template <class P>
struct ThetaAcc {
  using C = typename P::C;
  using T = typename P::T;
  typename P::Store* S;
  C* ov;           // buffer of the lone circle
  const T* g;      // multipliers f(|l|)/M, l = 0..Ntheta (shared memory)
  int ld, Nth, h, M, nseq;
  bool lone;       // Nphi/2 odd: the last sequence holds circle h-1 alone
  bool odd;        // parity a = 1

  __device__ __forceinline__ bool is_lone(int b) const { return lone && b == nseq - 1; }
  // home of complex slot n of sequence b: row and first column of the value pair
  __device__ __forceinline__ int home(int b, int n) const {
    return n < Nth ? n * ld + 2 * b : (n - Nth) * ld + 2 * b + h;
  }
  __device__ __forceinline__ C slot_ld(int b, int n) const {
    if (is_lone(b)) return ov[n];
    const int o = home(b, n);
    return C{P::ld(S + o), P::ld(S + o + 1)};
  }
  __device__ __forceinline__ void slot_st(int b, int n, C v) const {
    if (is_lone(b)) {
      ov[n] = v;
      return;
    }
    const int o = home(b, n);
    P::st(S + o, v.re);
    P::st(S + o + 1, v.im);
  }
  // circle sample q of the sequence: slot pi(q) with the parity sign for q >= Ntheta
  __device__ __forceinline__ C gather(int b, int q) const {
    const bool up = q < Nth;
    const int n = up ? q : 3 * Nth - 1 - q;
    C v;
    if (is_lone(b)) {
      v = C{P::ld(S + home(b, n)), P::zero()};
    } else {
      v = slot_ld(b, n);
    }
    if (!up && odd) v = Cx<P>::neg(v);
    return v;
  }
  __device__ __forceinline__ void scatter(int b, int q, C v) const {
    const bool up = q < Nth;
    const int n = up ? q : 3 * Nth - 1 - q;
    if (!up && odd) v = Cx<P>::neg(v);
    if (is_lone(b)) {
      P::st(S + home(b, n), v.re);
      return;
    }
    const int o = home(b, n);
    P::st(S + o, v.re);
    P::st(S + o + 1, v.im);
  }
  __device__ __forceinline__ T mult(int, int l) const { return g[l <= Nth ? l : M - l]; }
  __device__ __forceinline__ bool general(int) const { return false; }
};

template <class P>
struct PhiAcc {
  using C = typename P::C;
  using T = typename P::T;
  typename P::Store* S;
  C* ov;            // buffer of the lone middle ring
  const int2* pairs;  // (j1, j2), j2 < 0 for the lone ring; bit 30 of j1 marks a general pair
  const void* gtab;   // multipliers f(|m|)/Nphi of this shell: [Ntheta][Nphi/2+1] (global)
  size_t gbase;
  int ld, N, hN, nh;

  __device__ __forceinline__ int j1(int b) const { return pairs[b].x & 0x3fffffff; }
  __device__ __forceinline__ int j2(int b) const { return pairs[b].y; }
  __device__ __forceinline__ bool general(int b) const { return (pairs[b].x >> 30) & 1; }
  __device__ __forceinline__ C slot_ld(int b, int n) const {
    const int q = j2(b);
    if (q < 0) return ov[n];
    const int o = (n < hN ? j1(b) : q) * ld + 2 * (n < hN ? n : n - hN);
    return C{P::ld(S + o), P::ld(S + o + 1)};
  }
  __device__ __forceinline__ void slot_st(int b, int n, C v) const {
    const int q = j2(b);
    if (q < 0) {
      ov[n] = v;
      return;
    }
    const int o = (n < hN ? j1(b) : q) * ld + 2 * (n < hN ? n : n - hN);
    P::st(S + o, v.re);
    P::st(S + o + 1, v.im);
  }
  __device__ __forceinline__ C gather(int b, int k) const {
    const int q = j2(b);
    return C{P::ld(S + j1(b) * ld + k), q >= 0 ? P::ld(S + q * ld + k) : P::zero()};
  }
  __device__ __forceinline__ void scatter(int b, int k, C v) const {
    const int q = j2(b);
    P::st(S + j1(b) * ld + k, v.re);
    if (q >= 0) P::st(S + q * ld + k, v.im);
  }
  __device__ __forceinline__ T ring_mult(int j, int m) const {
    return P::from_tab(gtab, gbase + (size_t)j * nh + (m <= hN ? m : N - m));
  }
  __device__ __forceinline__ T mult(int b, int m) const { return ring_mult(j1(b), m); }
};

// ------------------------------------------------------------------ register-staged stage

enum { kFirst = 1, kLast = 2, kMul = 4 };

template <class P, class Acc, int R, int DIR, int MODE>
__device__ __forceinline__ void stage(const Acc& A, int N, int B, int Ns, const typename P::C* tw,
                                      const Consts<P>& k) {
  using C = typename P::C;
  using X = Cx<P>;
  constexpr int MAXI = (kMaxV + R - 1) / R;
  const int NR = N / R;
  const int total = B * NR;
  const int tws = N / (Ns * R);
  C v[MAXI][R];
#pragma unroll
  for (int u = 0; u < MAXI; ++u) {
    const int w = threadIdx.x + u * blockDim.x;
    if (w < total) {
      const int b = w / NR, j = w - b * NR;
      const int kk = j % Ns;
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const int n = j + t * NR;
        C x = (MODE & kFirst) ? A.gather(b, n) : A.slot_ld(b, n);
        if (MODE & kMul) {
          if (!A.general(b)) x = X::scale(x, A.mult(b, n));
        }
        v[u][t] = x;
      }
      if (Ns > 1) {
#pragma unroll
        for (int t = 1; t < R; ++t) {
          C wt = tw[t * kk * tws];
          if (DIR > 0) wt = X::conj_tw(wt);
          v[u][t] = P::cmul(v[u][t], wt);
        }
      }
      Dft<P, R, DIR>::run(v[u], k);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < MAXI; ++u) {
    const int w = threadIdx.x + u * blockDim.x;
    if (w < total) {
      const int b = w / NR, j = w - b * NR;
      const int kk = j % Ns;
      const int base = (j / Ns) * Ns * R + kk;
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (MODE & kLast) A.scatter(b, base + t * Ns, v[u][t]);
        else A.slot_st(b, base + t * Ns, v[u][t]);
      }
    }
  }
  __syncthreads();
}

// Generic lengths: each stage is its own function, so the register allocation of one radix does not
// weigh on the others (the call costs a register save and restore per stage).
template <class P, class Acc, int R, int DIR, int MODE>
__device__ __noinline__ void stage_ni(const Acc& A, int N, int B, int Ns, const typename P::C* tw,
                                      const Consts<P>& k) {
  stage<P, Acc, R, DIR, MODE>(A, N, B, Ns, tw, k);
}

template <class P, class Acc, int DIR, int MODE>
__device__ __forceinline__ void stage_r(int R, const Acc& A, int N, int B, int Ns, const typename P::C* tw,
                                        const Consts<P>& k) {
  switch (R) {
    case 8: stage_ni<P, Acc, 8, DIR, MODE>(A, N, B, Ns, tw, k); break;
    case 4: stage_ni<P, Acc, 4, DIR, MODE>(A, N, B, Ns, tw, k); break;
    case 2: stage_ni<P, Acc, 2, DIR, MODE>(A, N, B, Ns, tw, k); break;
    default: stage_ni<P, Acc, 3, DIR, MODE>(A, N, B, Ns, tw, k); break;
  }
}

// Exact two-real-sequence multiply for pairs whose rings have different multipliers:
// W_m = (f1+f2)/2 Z_m + (f1-f2)/2 conj(Z_{N-m}), on the spectrum held in the slots.
template <class P>
__device__ void general_multiply(const PhiAcc<P>& A, int B) {
  using C = typename P::C;
  const int nh = A.N / 2 + 1;
  C zm, zn, wm, wn;
  int b = -1, m = 0;
  // at most one (pair, m) per thread per round; pairs needing this are rare
  for (int base = 0; base < B * nh; base += blockDim.x) {
    const int w = base + threadIdx.x;
    bool act = false;
    if (w < B * nh) {
      b = w / nh;
      m = w - b * nh;
      act = A.general(b);
      if (act) {
        const int mn = (A.N - m) % A.N;
        zm = A.slot_ld(b, m);
        zn = A.slot_ld(b, mn);
        const auto f1 = A.ring_mult(A.j1(b), m), f2 = A.ring_mult(A.j2(b), m);
        const auto ca = P::half(P::add(f1, f2)), cd = P::half(P::sub(f1, f2));
        // conj(z) * cd: (re cd, -im cd)
        wm = C{P::add(P::mul(zm.re, ca), P::mul(zn.re, cd)), P::sub(P::mul(zm.im, ca), P::mul(zn.im, cd))};
        wn = C{P::add(P::mul(zn.re, ca), P::mul(zm.re, cd)), P::sub(P::mul(zn.im, ca), P::mul(zm.im, cd))};
      }
    }
    __syncthreads();
    if (act) {
      const int mn = (A.N - m) % A.N;
      A.slot_st(b, m, wm);
      if (mn != m) A.slot_st(b, mn, wn);
    }
    __syncthreads();
  }
}

template <class P>
__device__ __forceinline__ void maybe_general_multiply(const ThetaAcc<P>&, int) {}
template <class P>
__device__ __forceinline__ void maybe_general_multiply(const PhiAcc<P>& A, int B) {
  general_multiply<P>(A, B);
}

template <class P, class Acc>
__device__ void filter_pass(const Acc& A, int N, int B, const Factors& f, const typename P::C* tw,
                            const Consts<P>& k, bool has_general) {
  // forward transform: first stage gathers the logical sequence
  int Ns = 1;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    if (s == 0) stage_r<P, Acc, -1, kFirst>(R, A, N, B, Ns, tw, k);
    else stage_r<P, Acc, -1, 0>(R, A, N, B, Ns, tw, k);
    Ns *= R;
  }
  if (has_general) maybe_general_multiply<P>(A, B);
  // inverse transform: first stage multiplies, last stage scatters
  Ns = 1;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    const bool first = s == 0, last = s == f.nst - 1;
    if (first && last) stage_r<P, Acc, 1, kMul | kLast>(R, A, N, B, Ns, tw, k);
    else if (first) stage_r<P, Acc, 1, kMul>(R, A, N, B, Ns, tw, k);
    else if (last) stage_r<P, Acc, 1, kLast>(R, A, N, B, Ns, tw, k);
    else stage_r<P, Acc, 1, 0>(R, A, N, B, Ns, tw, k);
    Ns *= R;
  }
}

// Fixed lengths: the radix sequence is known at compile time and every stage is inlined.
template <class P, class Acc, int DIR, int MODE0, int R0, int... Rs>
__device__ __forceinline__ void run_stages(const Acc& A, int N, int B, int Ns, const typename P::C* tw,
                                           const Consts<P>& k) {
  constexpr bool last = sizeof...(Rs) == 0;
  constexpr int MODE = MODE0 | ((DIR > 0 && last) ? kLast : 0);
  stage<P, Acc, R0, DIR, MODE>(A, N, B, Ns, tw, k);
  if constexpr (!last) run_stages<P, Acc, DIR, 0, Rs...>(A, N, B, Ns * R0, tw, k);
}

template <class P, class Acc, int... Rs>
__device__ __forceinline__ void pass_ct(const Acc& A, int N, int B, const typename P::C* tw, const Consts<P>& k,
                                        bool has_general) {
  run_stages<P, Acc, -1, kFirst, Rs...>(A, N, B, 1, tw, k);
  if (has_general) maybe_general_multiply<P>(A, B);
  run_stages<P, Acc, 1, kMul, Rs...>(A, N, B, 1, tw, k);
}

// Lengths with a compiled radix sequence (theta circles of 2 Ntheta = Nphi = LEN).
template <int LEN>
struct FixedLen {
  static constexpr bool ok = LEN == 32 || LEN == 64 || LEN == 96 || LEN == 128 || LEN == 192 || LEN == 256;
};

template <class P, class Acc, int LEN>
__device__ __forceinline__ void pass_fixed(const Acc& A, int B, const typename P::C* tw, const Consts<P>& k,
                                           bool g) {
  if constexpr (LEN == 32) pass_ct<P, Acc, 8, 4>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 64) pass_ct<P, Acc, 8, 8>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 96) pass_ct<P, Acc, 8, 4, 3>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 128) pass_ct<P, Acc, 8, 8, 2>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 192) pass_ct<P, Acc, 8, 8, 3>(A, LEN, B, tw, k, g);
  else if constexpr (LEN == 256) pass_ct<P, Acc, 8, 8, 4>(A, LEN, B, tw, k, g);
}

template <class P, class Acc, int LEN>
__device__ __forceinline__ void run_pass(const Acc& A, int N, int B, const Factors& f, const typename P::C* tw,
                                         const Consts<P>& k, bool g) {
  if constexpr (LEN != 0) pass_fixed<P, Acc, LEN>(A, B, tw, k, g);
  else filter_pass<P>(A, N, B, f, tw, k, g);
}

// ------------------------------------------------------------------ kernel

template <class P>
struct Layout {
  typename P::Store* S;
  typename P::C* ov;
  typename P::C* tw_th;
  typename P::C* tw_ph;
  typename P::T* g_th;
  int2* pairs;
  int* misc;  // [0] pair count, [1] general flag, [2] block max exponent
};

template <class P>
__device__ Layout<P> carve(const ShellArgs2& A, unsigned char* base) {
  Layout<P> L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off = (off + bytes + 15) / 16 * 16;
    return p;
  };
  L.S = reinterpret_cast<typename P::Store*>(take(sizeof(typename P::Store) * (size_t)A.Nth * A.ldS));
  L.ov = reinterpret_cast<typename P::C*>(take(sizeof(typename P::C) * (size_t)max(2 * A.Nth, A.Nph)));
  L.tw_th = reinterpret_cast<typename P::C*>(take(sizeof(typename P::C) * 2 * (size_t)A.Nth));
  L.tw_ph = reinterpret_cast<typename P::C*>(take(sizeof(typename P::C) * (size_t)A.Nph));
  L.g_th = reinterpret_cast<typename P::T*>(take(sizeof(typename P::T) * (size_t)(A.Nth + 1)));
  L.pairs = reinterpret_cast<int2*>(take(sizeof(int2) * (size_t)(A.Nth / 2 + 1)));
  L.misc = reinterpret_cast<int*>(take(sizeof(int) * 4));
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

template <class P, int LEN>
__global__ void __launch_bounds__(512, 1) shell_kernel(ShellArgs2 A, LaunchIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using T = typename P::T;
  using C = typename P::C;
  const Layout<P> L = carve<P>(A, smem_raw);
  // i-major order: the fields of one radius run together, so their multiplier rows stay in L2
  const int i = blockIdx.x / A.nvars, v = blockIdx.x - i * A.nvars;
  const int shell = v * A.Nr + i;
  const VarInfo vi = A.var[v];
  const int Nth = A.Nth, Nph = A.Nph, ld = A.ldS;
  const int npts = Nth * Nph;
  constexpr bool dfp = std::is_same<P, DF>::value;

  // every stage must fit the registers: B * N <= blockDim * (R * floor(16 / R)) for each radix
  if (threadIdx.x == 0 && (int)blockDim.x < A.min_threads) atomicCAS(A.status, 0u, (unsigned)SPH_EDEVICE);
  if ((int)blockDim.x < A.min_threads) return;

  // twiddles, constants, theta multipliers
  const C* twth_g = static_cast<const C*>(A.tw_th);
  const C* twph_g = static_cast<const C*>(A.tw_ph);
  for (int n = threadIdx.x; n < 2 * Nth; n += blockDim.x) L.tw_th[n] = twth_g[n];
  for (int n = threadIdx.x; n < Nph; n += blockDim.x) L.tw_ph[n] = twph_g[n];
  const size_t gth_base = ((size_t)vi.cls * A.Nr + i) * (Nth + 1);
  for (int n = threadIdx.x; n <= Nth; n += blockDim.x) L.g_th[n] = P::from_tab(A.g_th, gth_base + n);
  Consts<P> K;
  K.c8 = P::from_tab(A.consts, 0);
  K.s3 = P::from_tab(A.consts, 1);

  // load the shell (raw FP64 first, so the compensated form can pick its scale)
  const double* srcd = static_cast<const double*>(io.in) + (size_t)shell * npts;
  const float* srcf = static_cast<const float*>(io.in) + (size_t)shell * npts;
  double* Sd = reinterpret_cast<double*>(L.S);
  unsigned emax = 0;
  for (int n = threadIdx.x; n < npts; n += blockDim.x) {
    const int j = n / Nph, k = n - j * Nph;
    double x = io.is_f32 ? (double)srcf[n] : srcd[n];
    if (io.map_in == kMapTanh) x = tanh(x);
    Sd[j * ld + k] = x;
    if (dfp) emax = max(emax, (unsigned)df_exp_field(x));
  }
  int E = 0;
  if (dfp) {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (threadIdx.x == 0) L.misc[2] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&L.misc[2], (int)emax);
    __syncthreads();
    E = L.misc[2] - 1023;
    for (int n = threadIdx.x; n < npts; n += blockDim.x) {
      const int j = n / Nph, k = n - j * Nph;
      P::st(L.S + j * ld + k, to_real<P>(Sd[j * ld + k], E));
    }
  }
  __syncthreads();

  const double lmax = A.lmax[vi.cls * A.Nr + i];
  const bool gauss = vi.kind == SPH_FILTER_GAUSS;
  const bool theta_on = gauss || lmax < (double)Nth;

  ThetaAcc<P> TA;
  TA.S = L.S;
  TA.ov = L.ov;
  TA.g = L.g_th;
  TA.ld = ld;
  TA.Nth = Nth;
  TA.h = Nph / 2;
  TA.M = 2 * Nth;
  TA.nseq = (Nph / 2 + 1) / 2;
  TA.lone = (Nph / 2) & 1;
  TA.odd = vi.parity != 0;

  // phi pairs: rings j and Ntheta-1-j, active unless both keep every mode
  const uint8_t* ring_info = A.ring_info + ((size_t)vi.cls * A.Nr + i) * Nth;
  if (threadIdx.x == 0) {
    int np = 0, gen = 0;
    for (int j = 0; j < (Nth + 1) / 2; ++j) {
      const int jj = Nth - 1 - j;
      const uint8_t a = ring_info[j], b = ring_info[jj];
      if (!((a | b) & 1)) continue;  // bit 0: ring active
      if (jj == j) {
        L.pairs[np++] = make_int2(j, -1);
      } else {
        const int g = (a >> 1) & 1;  // bit 1: multipliers of j and its mirror differ
        gen |= g;
        L.pairs[np++] = make_int2(j | (g << 30), jj);
      }
    }
    L.misc[0] = np;
    L.misc[1] = gen;
  }
  PhiAcc<P> PA;
  PA.S = L.S;
  PA.ov = L.ov;
  PA.pairs = L.pairs;
  PA.gtab = A.g_ph;
  PA.gbase = ((size_t)vi.cls * A.Nr + i) * (size_t)Nth * (Nph / 2 + 1);
  PA.ld = ld;
  PA.N = Nph;
  PA.hN = Nph / 2;
  PA.nh = Nph / 2 + 1;
  __syncthreads();
  const int npairs = L.misc[0];
  const bool has_general = L.misc[1] != 0;

  // filter: theta pass then phi pass, or the reverse order for the transpose
  for (int step = 0; step < 2; ++step) {
    if ((step == 0) != (io.transpose != 0)) {
      if (theta_on) run_pass<P, ThetaAcc<P>, LEN>(TA, 2 * Nth, TA.nseq, A.f_th, L.tw_th, K, false);
    } else {
      if (npairs) run_pass<P, PhiAcc<P>, LEN>(PA, Nph, npairs, A.f_ph, L.tw_ph, K, has_general);
    }
  }

  const size_t off = (size_t)shell * npts;
  for (int n = threadIdx.x; n < npts; n += blockDim.x) {
    const int j = n / Nph, k = n - j * Nph;
    double y = from_real<P>(P::ld(L.S + j * ld + k), E);
    if (io.map_out == kOutTanhGrad) {
      const double z = io.is_f32 ? (double)static_cast<const float*>(io.aux)[off + n]
                                 : static_cast<const double*>(io.aux)[off + n];
      const double t = tanh(z);
      y *= (1.0 - t * t);
    }
    if (io.is_f32) static_cast<float*>(io.out)[off + n] = (float)y;
    else static_cast<double*>(io.out)[off + n] = y;
  }
}

template <class P>
size_t shell_smem(const ShellArgs2& a) {
  auto up = [](size_t x) { return (x + 15) / 16 * 16; };
  const size_t cs = 2 * sizeof(typename P::T);
  size_t s = up(sizeof(typename P::Store) * (size_t)a.Nth * a.ldS);
  s += up(cs * (size_t)std::max(2 * a.Nth, a.Nph));
  s += up(cs * 2 * (size_t)a.Nth);
  s += up(cs * (size_t)a.Nph);
  s += up(sizeof(typename P::T) * (size_t)(a.Nth + 1));
  s += up(sizeof(int2) * (size_t)(a.Nth / 2 + 1));
  s += up(sizeof(int) * 4);
  return s;
}

template <class P, int LEN>
cudaError_t launch_impl(const ShellArgs2& a, int threads, size_t smem, const LaunchIO& io, cudaStream_t s) {
  const dim3 grid((unsigned)(a.nvars * a.Nr));
  shell_kernel<P, LEN><<<grid, threads, smem, s>>>(a, io);
  return cudaGetLastError();
}

template <class P, int LEN>
cudaError_t set_attr_impl(int bytes) {
  return cudaFuncSetAttribute(shell_kernel<P, LEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class P>
size_t smem_impl(const ShellArgs2& a) {
  return shell_smem<P>(a);
}

}  // namespace shellk
}  // namespace sph
