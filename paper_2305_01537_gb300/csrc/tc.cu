// Split-precision tensor-core form of the double FFT filter (SPH_PREC_SPLIT_TC).
//
// Each pass of Sec. II.C is a real, symmetric, circulant operator on a vector of length L: a
// doubled great circle (L = 2 Ntheta, with the field's parity sign across the pole) for the theta
// pass, a ring (L = Nphi) for the phi pass. Only the removed part H c = c - M c is computed here,
// with H = F^-1 diag(1 - f) F, and the pass writes c - H c in FP64. The DFT F and its inverse are
// dense matrices shared by every vector of a length, so they run as tcgen05 GEMMs over 128 vectors
// at a time; the per-vector multipliers 1 - f(|m|, cutoff) are applied between the two GEMMs.
//
// Real DFT split (exact algebra, no approximation): with H = L/2, u_q = c_q + c_{L-q}
// (u_0 = c_0, u_H = c_H) and v_q = c_q - c_{L-q},
//   X_c[m] = sum_{q=0}^{H} u_q cos(2 pi m q / L),            m = 0 .. H
//   X_s[m] = sum_{q=1}^{H-1} v_q sin(2 pi m q / L),          m = 1 .. H-1
//   y_e[k] = (1/L) sum_{m=0}^{H} w_m h_m X_c[m] cos(2 pi m k / L),  w_0 = w_H = 1, else 2
//   y_o[k] = (2/L) sum_{m=1}^{H-1} h_m X_s[m] sin(2 pi m k / L)
//   (H c)_k = y_e[k] + y_o[k],  (H c)_{L-k} = y_e[k] - y_o[k].
// Four GEMMs (CF, SF, CI, SI) with at most H outputs each; the Nyquist terms X_c[H] and y_e[H]
// (alternating sums) are summed exactly in 64-bit integers on the CUDA cores.
//
// Exact products from BF16 (Ozaki-style splitting): every operand value v, scaled by a power of two
// so that |v| <= 1/2, is written as six balanced base-256 digits, v = sum_a d_a 256^-(a+1) with
// |d_a| <= 128, each slice d_a 256^-(a+1) exact in BF16. A slice-pair product is exact. The tensor
// core adds the products of one MMA and the accumulator after aligning them to the largest one and
// truncating, so the sums are exact only while every addend is an integer in the accumulator's
// unit and the total stays below 2^24 units: each diagonal a + b = t (t = 0..5, all pairs of one
// scale, at most 6 x 129 x 2^14 < 2^24 units for K <= 160) therefore has an accumulator of its
// own. Pairs with a + b >= 6 are dropped (2^-48 of the result). The six accumulators are summed in
// compensated FP32 pairs, then converted to FP64 with integer operations.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "df32.h"
#include "internal.h"

namespace sph {
namespace tcx {

constexpr int kM = 128;            // vectors per tile (MMA M)
constexpr int kKC = 32;            // K values per pipeline chunk (two MMA K-steps of 16)
constexpr int kS = 6;              // slices per operand
constexpr int kAcc = 6;            // accumulators: one per diagonal a + b = 0 .. 5
constexpr int kMaxNPh = 80;        // GEMM N per launch of the K loop (6 x 80 <= 512 TMEM columns)
constexpr int kMaxL = 256;
constexpr uint32_t kStageA = kS * kM * kKC * 2;       // 49152 bytes
constexpr uint32_t kStageB = kS * kMaxNPh * kKC * 2;  // 30720 bytes
constexpr uint32_t kStage = kStageA + kStageB;        // 79872 bytes (a multiple of 1024)
constexpr int kThr = 512;          // threads per CTA (4 warps per tensor-memory lane quarter)
constexpr long long kWaitLimit = 1LL << 20;           // bounded mbarrier polls (seconds at most)

enum Op { kCF = 0, kSF = 1, kCI = 2, kSI = 3 };

// Offset (elements) of (row, k) in a ROWS x kKC operand chunk stored K-major without swizzle:
// 8-row x 8-element core matrices of 128 contiguous bytes; LBO (next core matrix along K) = 128 B,
// SBO (next group of 8 rows) = (kKC / 8) * 128 B. Rows [8g, 8g + 8) are contiguous.
__host__ __device__ inline uint32_t kmaj_elem(int row, int k) {
  return (uint32_t)((row >> 3) * (kKC / 8) * 64 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7));
}

struct OpTab {
  const uint16_t* tab;  // [KP / kKC][kS][NP][kKC] BF16 slices, core-matrix layout per (chunk, slice)
  int N, K;             // valid output and reduction sizes
  int NPh, nh;          // outputs per pass of the K loop (multiple of 16) and passes; NP = NPh * nh
  int KP;               // padded K (multiple of kKC)
};

struct TcArgs {
  int pass;                 // 0: theta (doubled circles), 1: phi (rings)
  int L;                    // vector length
  int Nr, Nth, Nph;
  const double* src;        // state read by the pass
  double* dst;              // state written (may equal src); only active vectors are written
  const int* list;          // theta: active shells v*Nr+i; phi: active rings (v*Nr+i)*Nth+j
  long long nvec;           // theta: entries * Nph/2; phi: entries
  const float2* h;          // 1 - f as FP32 pairs: theta [ncls][Nr][Nth+1]; phi [ncls][Nr][Nth][Nph/2+1]
  const VarInfo* var;
  OpTab op[4];
  int Ef, Ei;               // operator scales: forward (CF, SF) = 2^Ef * slices, inverse 2^Ei
  float2* scratch;          // per CTA: Yc [kM][H+1], Ys [kM][H-1], ye [kM][H+1]
  uint4* akeep;             // per CTA: the A stages of a GEMM's first output half, [KP / kKC][kStageA / 16]
  int akeep_chunks;         // chunks per CTA in akeep (0 when no GEMM has two output halves)
  unsigned* status;
};

struct Row {
  size_t base;              // offset of element 0 of the vector in the state
  const float2* h;          // multipliers of the vector's modes 0 .. H
  int neg;                  // theta: second half carries the parity sign -1
  int ex;                   // input scale exponent
  int ey;                   // spectrum scale exponent
  int valid;
};

struct Smem {
  Row row[kM];
  int emax[kM];                // biased exponent maxima (FP64 input, FP32 spectrum)
  unsigned long long nyq[kM];  // exact Nyquist sums (two's complement) of the CF and CI operands
  unsigned long long bar[2];
  uint32_t tslot;
  int abort;
};

constexpr uint32_t kSmemBytes = 2 * kStage + ((sizeof(Smem) + 127) / 128) * 128;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;                 // LBO: next core matrix along K
  d |= (uint64_t)(((kKC / 8) * 128) >> 4) << 32;   // SBO: next group of 8 rows
  d |= (uint64_t)1 << 46;                          // descriptor version
  return d;                                        // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128.
__device__ __forceinline__ uint32_t make_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// v * 2^(48 - E) rounded to an integer (|result| < 2^47 when |v| < 2^(E-1)).
__device__ __forceinline__ long long fx64(double d, int E) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  const int sh = 1027 + E - e;
  if (e == 0 || sh >= 62) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const long long t = sh >= 1 ? ((m >> (sh - 1)) + 1) >> 1 : (1LL << 47) - 1;  // sh < 1 cannot occur for a valid E
  return b < 0 ? -t : t;
}
__device__ __forceinline__ long long fx32(float f, int E) {
  const int b = __float_as_int(f);
  const int e = (b >> 23) & 0xFF;
  const int sh = 102 + E - e;
  if (e == 0 || sh >= 40) return 0;
  const long long m = (long long)((b & 0x7FFFFF) | 0x800000);
  const long long t = sh >= 1 ? ((m >> (sh - 1)) + 1) >> 1 : (sh > -24 ? (m << (-sh)) : (1LL << 47) - 1);
  return b < 0 ? -t : t;
}

// Six BF16 slices of eight fixed-point values: slice a holds d_a 256^-(a+1), the balanced digits
// of t 2^-48 (t + 0x808080808080 has base-256 digits d_a + 128; the top one is not masked, so it
// may be 256 when |t| approaches 2^47). Each slice value is built exactly from its byte: the float
// with exponent field 150 - 8(a+1) and the byte as low mantissa bits is (2^23 + byte) 2^-8(a+1).
__device__ __forceinline__ void slice8(const long long t[8], uint4 out[kS]) {
  uint32_t w[kS][4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float f[kS][2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const long long tb = t[2 * p + hh] + 0x808080808080LL;
      const uint32_t lo = (uint32_t)tb, hi = (uint32_t)(tb >> 32);
      const uint32_t byte[kS] = {hi >> 8, hi & 0xFFu, lo >> 24, (lo >> 16) & 0xFFu, (lo >> 8) & 0xFFu, lo & 0xFFu};
#pragma unroll
      for (int a = 0; a < kS; ++a) {
        const int ef = 150 - 8 * (a + 1);
        f[a][hh] = __fsub_rn(__int_as_float((ef << 23) | (int)byte[a]), __int_as_float((ef << 23) | 128));
      }
    }
#pragma unroll
    for (int a = 0; a < kS; ++a) {
      const __nv_bfloat162 v = __floats2bfloat162_rn(f[a][0], f[a][1]);
      w[a][p] = *reinterpret_cast<const uint32_t*>(&v);
    }
  }
#pragma unroll
  for (int a = 0; a < kS; ++a) out[a] = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
}

// Compensated FP32 pair helpers (Knuth TwoSum, FMA-based exact product).
__device__ __forceinline__ df df_renorm(float s, float e) {
  const float hi = __fadd_rn(s, e);
  return df{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
// D0 + ... + D5 (each exact; D_t is about 2^-8t of D0): the leading three summed without error,
// the tail (below 2^-24 of the result) with ordinary additions.
__device__ __forceinline__ df combine6(const float d[kAcc]) {
  const df s = two_sum(d[0], d[1]);
  const df a = two_sum(s.lo, d[2]);
  const float tail = __fadd_rn(a.lo, __fadd_rn(d[3], __fadd_rn(d[4], d[5])));
  const df f = two_sum(s.hi, a.hi);
  return df_renorm(f.hi, __fadd_rn(f.lo, tail));
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_renorm(p, e);
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return df_renorm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

// Offset of element q of a vector: theta circles run down meridian k, then back up meridian
// k + Nphi/2 (Sec. II.C double covering); rings are contiguous.
__device__ __forceinline__ size_t elem(const TcArgs& A, size_t base, int q) {
  if (A.pass == 0)
    return q < A.Nth ? base + (size_t)q * A.Nph : base + (size_t)(2 * A.Nth - 1 - q) * A.Nph + A.Nph / 2;
  return base + q;
}
// The parity sign of element q applies (theta circles of odd fields, second half).
__device__ __forceinline__ bool flip(const TcArgs& A, const Row& R, int q) { return R.neg && q >= A.Nth; }
// Element q as a fixed-point integer at scale E (the sign applied to the integer).
__device__ __forceinline__ long long load_fx(const TcArgs& A, const Row& R, int q, int E) {
  const long long t = fx64(A.src[elem(A, R.base, q)], E);
  return flip(A, R, q) ? -t : t;
}
// Writes c_q - hc for element q: the stored value is s (c_q - hc) = x_stored - s hc with s the
// parity sign, so the sign goes on hc with an integer operation and one FP64 subtraction remains.
__device__ __forceinline__ void update_c(const TcArgs& A, const Row& R, int q, double hc) {
  const size_t o = elem(A, R.base, q);
  const long long sb = flip(A, R, q) ? (long long)0x8000000000000000ULL : 0LL;
  A.dst[o] = A.src[o] - __longlong_as_double(__double_as_longlong(hc) ^ sb);
}

struct Ctx {
  const TcArgs& A;
  Smem& S;
  unsigned char* stage;
  uint32_t tmem;
  float2* Yc;   // [kM][H+1]: h X_c[m], m = 0 .. H
  float2* Ys;   // [kM][H-1]: h X_s[m + 1]
  float2* Ye;   // [kM][H+1]: y_e[k]
  uint4* akeep; // this CTA's copies of the first half's A stages
  unsigned G;   // chunks issued so far by this CTA
};

// Eight consecutive K values of GEMM operand A (vector data) for row r, as fixed-point integers;
// *nyq gets their contribution to the Nyquist sum of the CF or CI operand.
__device__ __forceinline__ void gather8(Ctx& C, int op, int r, int k0, long long t[8], long long* nyq) {
  const TcArgs& A = C.A;
  const Row& R = C.S.row[r];
  const int L = A.L, H = L / 2;
  *nyq = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t[i] = 0;
  if (!R.valid) return;
  if (op == kCF) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = k0 + i;
      if (q <= H) {
        long long u = load_fx(A, R, q, R.ex);
        if (q != 0 && q != H) u += load_fx(A, R, L - q, R.ex);
        t[i] = u;
        *nyq += (q & 1) ? -u : u;  // cos(pi q)
      }
    }
  } else if (op == kSF) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = k0 + i + 1;
      if (q < H) t[i] = load_fx(A, R, q, R.ex) - load_fx(A, R, L - q, R.ex);
    }
  } else {
    const float2* src = op == kCI ? C.Yc + (size_t)r * (H + 1) : C.Ys + (size_t)r * (H - 1);
    const int K = op == kCI ? H + 1 : H - 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = k0 + i;
      if (m < K) {
        const float2 y = src[m];
        t[i] = fx32(y.x, R.ey) + fx32(y.y, R.ey);
        if (op == kCI) {
          const long long wt = (m == 0 || m == H) ? t[i] : 2 * t[i];  // w_m cos(pi m)
          *nyq += (m & 1) ? -wt : wt;
        }
      }
    }
  }
}

// One pass of the K loop of a GEMM over 128 vectors for outputs [half NPh, (half + 1) NPh):
// accumulator t (diagonal a + b = t) in tensor-memory columns [t NPh, (t + 1) NPh). Returns false
// if a wait ran out.
__device__ bool gemm(Ctx& C, int op, int half) {
  const TcArgs& A = C.A;
  const OpTab& T = A.op[op];
  const int nk = T.KP / kKC;
  const int NP = T.NPh * T.nh;
  const int tid = threadIdx.x;
  const uint32_t idesc = make_idesc(T.NPh);
  bool init[kAcc] = {false, false, false, false, false, false};
  for (int kc = 0; kc < nk; ++kc) {
    const unsigned G = C.G++;
    const int s = (int)(G & 1u);
    unsigned char* sa = C.stage + (size_t)s * kStage;
    unsigned char* sb = sa + kStageA;
    // stage s is free once the MMAs of chunk G - 2 are done; each thread waits by itself (no block
    // barrier here, so the warps that do not issue MMAs start this chunk during the issue), and a
    // wait that runs out is acted on at the barrier below
    const bool waited = G < 2 || mbar_wait(su32(&C.S.bar[s]), ((G - 2) >> 1) & 1u);
    // operand A: six slices of the vector data. A GEMM with two output halves produces them in
    // its first half and keeps a copy; the second half copies the stage back instead.
    uint4* keep = T.nh > 1 ? C.akeep + (size_t)kc * (kStageA / 16) : nullptr;
    if (half == 0) {
      for (int task = tid; task < kM * (kKC / 8); task += kThr) {
        const int r = task & (kM - 1), g = task / kM;
        long long t[8], nyq;
        gather8(C, op, r, kc * kKC + g * 8, t, &nyq);
        if (nyq != 0) atomicAdd(&C.S.nyq[r], (unsigned long long)nyq);
        uint4 w[kS];
        slice8(t, w);
#pragma unroll
        for (int a = 0; a < kS; ++a) {
          const uint32_t o = a * kM * kKC * 2 + 2 * kmaj_elem(r, g * 8);
          *reinterpret_cast<uint4*>(sa + o) = w[a];
          if (keep) keep[o / 16] = w[a];
        }
      }
    } else {
      for (int i = tid; i < (int)(kStageA / 16); i += kThr) reinterpret_cast<uint4*>(sa)[i] = keep[i];
    }
    // operand B: the chunk's six operator slices, rows of this half (contiguous 8-row groups)
    {
      const int per_slice = T.NPh * kKC * 2 / 16;
      for (int i = tid; i < kS * per_slice; i += kThr) {
        const int b = i / per_slice, j = i - b * per_slice;
        const uint4* src = reinterpret_cast<const uint4*>(T.tab + ((size_t)(kc * kS + b) * NP + half * T.NPh) * kKC);
        reinterpret_cast<uint4*>(sb + (size_t)b * T.NPh * kKC * 2)[j] = __ldg(src + j);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(waited ? 1 : 0)) return false;
    if (tid == kThr - 32) {  // lane 0 of the last warp issues the chunk's MMAs
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = su32(sa), b0 = su32(sb);
#pragma unroll
      for (int ks = 0; ks < kKC / 16; ++ks) {
#pragma unroll
        for (int a = 0; a < kS; ++a) {
#pragma unroll
          for (int b = 0; a + b < kAcc; ++b) {
            const int acc = a + b;
            const uint32_t d = C.tmem + (uint32_t)(acc * T.NPh);
            const uint64_t da = make_desc(a0 + (uint32_t)(a * kM * kKC * 2 + ks * 256));
            const uint64_t db = make_desc(b0 + (uint32_t)(b * T.NPh * kKC * 2 + ks * 256));
            const uint32_t en = init[acc] ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                "l"(da), "l"(db), "r"(idesc), "r"(en));
            init[acc] = true;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&C.S.bar[s]))
                   : "memory");
    }
  }
  // wait for the last chunk (its commit covers every earlier MMA of this thread)
  const unsigned last = C.G - 1;
  if (!__syncthreads_and(mbar_wait(su32(&C.S.bar[last & 1u]), (last >> 1) & 1u) ? 1 : 0)) return false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

// Eight columns of the six accumulators for this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld6(uint32_t taddr, int NPh, float d[kAcc][8]) {
  uint32_t v[kAcc][8];
#pragma unroll
  for (int acc = 0; acc < kAcc; ++acc)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[acc][0]), "=r"(v[acc][1]), "=r"(v[acc][2]), "=r"(v[acc][3]), "=r"(v[acc][4]),
                   "=r"(v[acc][5]), "=r"(v[acc][6]), "=r"(v[acc][7])
                 : "r"(taddr + (uint32_t)(acc * NPh)));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int acc = 0; acc < kAcc; ++acc)
#pragma unroll
    for (int i = 0; i < 8; ++i) d[acc][i] = __uint_as_float(v[acc][i]);
}

// Epilogue of one pass of a GEMM. Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (one vector
// each) and the 8-column groups w / 4, w / 4 + 4, ... of the pass's output columns.
__device__ void epilogue(Ctx& C, int op, int half) {
  const TcArgs& A = C.A;
  const OpTab& T = A.op[op];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, side = warp >> 2;
  const int r = 32 * quarter + lane;
  const Row& R = C.S.row[r];
  const int L = A.L, H = L / 2;
  const uint32_t taddr = C.tmem + ((uint32_t)(32 * quarter) << 16);
  const int c_begin = side * 8, c_end = T.NPh, c_step = (kThr / 128) * 8;
  const int S2 = R.ex + A.Ef + R.ey + A.Ei;  // output scale of the inverse GEMMs
  int emax = 0;
  for (int c0 = c_begin; c0 < c_end; c0 += c_step) {
    float d[kAcc][8];
    tmem_ld6(taddr + (uint32_t)c0, T.NPh, d);
    if (!R.valid) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int n = half * T.NPh + c0 + i;
      if (n >= T.N) continue;
      float dd[kAcc];
#pragma unroll
      for (int acc = 0; acc < kAcc; ++acc) dd[acc] = d[acc][i];
      const df z = combine6(dd);
      if (op == kCF || op == kSF) {
        const int m = op == kCF ? n : n + 1;
        const float2 hm = R.h[m];
        const df y = df_mul(z, df{hm.x, hm.y});
        const float2 yv = make_float2(y.hi, y.lo);
        if (op == kCF) C.Yc[(size_t)r * (H + 1) + n] = yv;
        else C.Ys[(size_t)r * (H - 1) + n] = yv;
        emax = max(emax, (__float_as_int(y.hi) >> 23) & 0xFF);
      } else if (op == kCI) {
        const int k = n;
        if (k == 0) update_c(A, R, 0, df_to_double(z, S2));
        else C.Ye[(size_t)r * (H + 1) + k] = make_float2(z.hi, z.lo);  // read by the SI epilogue
      } else {
        const int k = n + 1;
        const float2 e = C.Ye[(size_t)r * (H + 1) + k];
        const df ye{e.x, e.y};
        const double hp = df_to_double(df_add(ye, z), S2);
        const double hm = df_to_double(df_add(ye, df_neg(z)), S2);
        update_c(A, R, k, hp);
        update_c(A, R, L - k, hm);
      }
    }
  }
  // Nyquist terms from the exact integer sums (one thread per vector, once per GEMM)
  if (side == 0 && half == 0 && R.valid && (op == kCF || op == kCI)) {
    const long long sum = (long long)C.S.nyq[r];
    if (op == kCF) {
      // X_c[H] in GEMM units: sum 2^-48 (data scale) 2^-Ef (operator scale)
      const df z = df_from_double((double)sum, 48 + A.Ef);
      const float2 hH = R.h[H];
      const df y = df_mul(z, df{hH.x, hH.y});
      C.Yc[(size_t)r * (H + 1) + H] = make_float2(y.hi, y.lo);
      emax = max(emax, (__float_as_int(y.hi) >> 23) & 0xFF);
    } else {
      // y_e[H] = (1/L) sum_m w_m cos(pi m) h_m X_c[m], in GEMM units 2^-48 2^-Ei
      const df z = df_from_double((double)sum / (double)L, 48 + A.Ei);
      update_c(A, R, H, df_to_double(z, S2));
    }
  }
  if (op == kCF || op == kSF) atomicMax(&C.S.emax[r], emax);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(kThr, 1) tc_pass_kernel(TcArgs A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  Smem& S = *reinterpret_cast<Smem*>(smem + 2 * kStage);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int L = A.L, H = L / 2;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tslot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    S.abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  Ctx C{A, S, smem, S.tslot, nullptr, nullptr, nullptr, nullptr, 0u};
  C.Yc = A.scratch + (size_t)kM * (3 * H + 1) * blockIdx.x;
  C.Ys = C.Yc + (size_t)kM * (H + 1);
  C.Ye = C.Ys + (size_t)kM * (H - 1);
  C.akeep = A.akeep + (size_t)A.akeep_chunks * (kStageA / 16) * blockIdx.x;
  const long long ntiles = (A.nvec + kM - 1) / kM;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    // vector set-up: row r <- vector tile * 128 + r
    if (tid < kM) {
      Row R{};
      const long long vg = tile * kM + tid;
      R.valid = vg < A.nvec;
      if (R.valid) {
        if (A.pass == 0) {
          const int half = A.Nph / 2;
          const int shell = A.list[vg / half];
          const int k = (int)(vg % half);
          const int v = shell / A.Nr, i = shell - v * A.Nr;
          const VarInfo vi = A.var[v];
          R.base = (size_t)shell * A.Nth * A.Nph + k;
          R.h = A.h + ((size_t)vi.cls * A.Nr + i) * (A.Nth + 1);
          R.neg = vi.parity;
        } else {
          const int ring = A.list[vg];
          const int j = ring % A.Nth, vi_ = ring / A.Nth;
          const int v = vi_ / A.Nr, i = vi_ - v * A.Nr;
          const VarInfo vi = A.var[v];
          R.base = (size_t)ring * A.Nph;
          R.h = A.h + (((size_t)vi.cls * A.Nr + i) * A.Nth + j) * (H + 1);
          R.neg = 0;
        }
      }
      S.row[tid] = R;
      S.emax[tid] = 0;
      S.nyq[tid] = 0ull;
    }
    __syncthreads();
    // input scale: largest FP64 exponent over the vector; lanes run along contiguous memory (the
    // vector index for theta circles, the ring for rings)
    if (A.pass == 0) {
      const int r = tid & (kM - 1), part = tid / kM, np = kThr / kM;
      const Row& R = S.row[r];
      int e = 0;
      if (R.valid)
        for (int q = part; q < L; q += np)
          e = max(e, (int)((__double_as_longlong(A.src[elem(A, R.base, q)]) >> 52) & 0x7FF));
      atomicMax(&S.emax[r], e);
    } else {
      const int lane = tid & 31;
      for (int r = warp; r < kM; r += kThr / 32) {
        const Row& R = S.row[r];
        int e = 0;
        if (R.valid)
          for (int q = lane; q < L; q += 32) e = max(e, (int)((__double_as_longlong(A.src[R.base + q]) >> 52) & 0x7FF));
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0) atomicMax(&S.emax[r], e);
      }
    }
    __syncthreads();
    if (tid < kM) {
      // |u| <= 2 max|c| < 2^(e - 1023 + 2), so E = e - 1023 + 3 keeps |u| 2^-E below 1/2
      S.row[tid].ex = S.emax[tid] ? S.emax[tid] - 1023 + 3 : 0;
      S.emax[tid] = 0;
    }
    __syncthreads();
    for (int op = kCF; op <= kSI && ok; ++op) {
      if (op == kCI) {
        __syncthreads();  // spectrum maxima complete
        if (tid < kM) {
          // |Y| < 2^(e - 126) for the largest FP32 exponent field e: E = e - 125 keeps |Y| 2^-E < 1/2
          S.row[tid].ey = S.emax[tid] ? S.emax[tid] - 125 : 0;
          S.nyq[tid] = 0ull;
        }
        __syncthreads();
      }
      if (op == kSI) __syncthreads();  // y_e complete before the SI epilogue reads it
      for (int half = 0; half < A.op[op].nh && ok; ++half) {
        ok = gemm(C, op, half);
        if (ok) epilogue(C, op, half);
      }
    }
    if (!ok) atomicExch(&S.abort, 1);
    __syncthreads();
    if (S.abort) {
      if (tid == 0) atomicCAS(A.status, 0u, (unsigned)SPH_ETIMEOUT);
      ok = false;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tslot), "r"(512));
}

// ---------------------------------------------------------------- host side

// Balanced base-256 digits of v (|v| <= 1/2), most significant first: v ~ sum_a d_a 256^-(a+1).
void digits(long double v, int d[kS]) {
  for (int a = 0; a < kS; ++a) {
    v *= 256.0L;
    const long double r = rintl(v);
    d[a] = (int)r;
    v -= r;
  }
}

uint16_t bf16_bits_exact(int d, int a) {
  const float f = ldexpf((float)d, -8 * (a + 1));  // at most 8 significant bits: exact in BF16
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

int pad_to(int n, int m) { return (n + m - 1) / m * m; }

// Slices of the N x K operator F(n, k) 2^-E in the layout gemm() reads.
template <class F>
std::vector<uint16_t> build_op(int N, int K, int E, F f, OpTab* t) {
  t->N = N;
  t->K = K;
  t->nh = 1;
  t->NPh = pad_to(std::max(N, 16), 16);
  if (t->NPh > kMaxNPh) {
    t->nh = 2;
    t->NPh = pad_to((N + 1) / 2, 16);
  }
  t->KP = pad_to(std::max(K, 1), kKC);
  const int NP = t->NPh * t->nh;
  std::vector<uint16_t> tab((size_t)(t->KP / kKC) * kS * NP * kKC, 0);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      int d[kS];
      digits(ldexpl(f(n, k), -E), d);
      const int kc = k / kKC;
      for (int b = 0; b < kS; ++b)
        tab[((size_t)kc * kS + b) * NP * kKC + kmaj_elem(n, k % kKC)] = bf16_bits_exact(d[b], b);
    }
  return tab;
}

}  // namespace tcx

struct TcPass {
  int L = 0;
  void* d_tab = nullptr;           // the four operators' slices
  tcx::OpTab op[4];
  int Ef = 0, Ei = 0;
  float2* d_h = nullptr;
  int* d_list = nullptr;
  std::vector<long long> var_off;  // list entries of fields [0, v): prefix counts
  std::vector<int> copy_runs;      // theta pass: [field, first shell, shells] runs of identity shells
};

// Scratch set 0 serves sph_filter_apply and the calls built on it; sets 1..3 (allocated on first
// use) serve the three streams of the host-buffer pipeline, whose chunk launches may overlap.
struct TcPlan {
  TcPass pass[2];
  float2* d_scratch = nullptr;       // set 0
  uint4* d_akeep = nullptr;
  float2* d_scratch_pipe = nullptr;  // sets 1..3
  uint4* d_akeep_pipe = nullptr;
  size_t scratch_set = 0, akeep_set = 0;  // elements per set
  int akeep_chunks = 0;
  int nsm = 0;
};

namespace {

sph_status build_pass(TcPass* P, int L) {
  using namespace tcx;
  const long double pi = acosl(-1.0L);
  const int H = L / 2;
  P->L = L;
  // forward entries are at most 1 -> E = 1; inverse entries at most 2/L -> smallest E with 2/L <= 2^(E-1)
  P->Ef = 1;
  int Ei = 1;
  while (ldexpl(1.0L, Ei - 2) >= 2.0L / (long double)L) --Ei;
  P->Ei = Ei;
  auto cs = [&](long long m, long long k) { return cosl(2.0L * pi * (long double)((m * k) % L) / (long double)L); };
  auto sn = [&](long long m, long long k) { return sinl(2.0L * pi * (long double)((m * k) % L) / (long double)L); };
  // the cos GEMMs leave out their Nyquist output (m = H, k = H), summed exactly in the kernel
  std::vector<uint16_t> t0 = build_op(H, H + 1, P->Ef, [&](int m, int q) { return cs(m, q); }, &P->op[kCF]);
  std::vector<uint16_t> t1 =
      build_op(H - 1, H - 1, P->Ef, [&](int n, int k) { return sn(n + 1, k + 1); }, &P->op[kSF]);
  std::vector<uint16_t> t2 = build_op(
      H, H + 1, P->Ei,
      [&](int k, int m) { return ((m == 0 || m == H) ? 1.0L : 2.0L) * cs(m, k) / (long double)L; }, &P->op[kCI]);
  std::vector<uint16_t> t3 =
      build_op(H - 1, H - 1, P->Ei, [&](int n, int k) { return 2.0L * sn(k + 1, n + 1) / (long double)L; }, &P->op[kSI]);
  const size_t total = t0.size() + t1.size() + t2.size() + t3.size();
  if (cudaMalloc(&P->d_tab, total * 2) != cudaSuccess) return SPH_ENOMEM;
  uint16_t* d = static_cast<uint16_t*>(P->d_tab);
  const std::vector<uint16_t>* ts[4] = {&t0, &t1, &t2, &t3};
  size_t off = 0;
  for (int o = 0; o < 4; ++o) {
    if (cudaMemcpy(d + off, ts[o]->data(), ts[o]->size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return SPH_ECUDA;
    P->op[o].tab = d + off;
    off += ts[o]->size();
  }
  return SPH_OK;
}

}  // namespace

sph_status tc_setup(sph_filter_plan_s* p) {
  const int Lth = 2 * p->Nth, Lph = p->Nph;
  if (Lth < 8 || Lph < 8 || Lth > tcx::kMaxL || Lph > tcx::kMaxL) return SPH_EUNSUPPORTED;
  TcPlan* T = new (std::nothrow) TcPlan();
  if (!T) return SPH_ENOMEM;
  p->tc = T;
  sph_status st = build_pass(&T->pass[0], Lth);
  if (st == SPH_OK) st = build_pass(&T->pass[1], Lph);
  if (st != SPH_OK) return st;
  const int Nr = p->Nr, Nth = p->Nth, Nph = p->Nph, ncls = p->ncls;
  // high-pass multipliers 1 - f (Sec. II.C filter functions) and the active vectors of each pass
  std::vector<float2> hth((size_t)ncls * Nr * (Nth + 1)), hph((size_t)ncls * Nr * Nth * (Nph / 2 + 1));
  auto pair = [](long double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (long double)hi));
  };
  for (int c = 0; c < ncls; ++c)
    for (int i = 0; i < Nr; ++i) {
      const long double lm = p->h_lmax[(size_t)c * Nr + i];
      for (int l = 0; l <= Nth; ++l)
        hth[((size_t)c * Nr + i) * (Nth + 1) + l] = pair(1.0L - filter_value(p->cls_kind[(size_t)c], l, lm));
      for (int j = 0; j < Nth; ++j) {
        const long double mm = p->h_mmax[((size_t)c * Nr + i) * Nth + j];
        for (int m = 0; m <= Nph / 2; ++m)
          hph[(((size_t)c * Nr + i) * Nth + j) * (Nph / 2 + 1) + m] =
              pair(1.0L - filter_value(p->cls_kind[(size_t)c], m, mm));
      }
    }
  std::vector<int> lth, lph;
  T->pass[0].var_off.assign(1, 0);
  T->pass[1].var_off.assign(1, 0);
  for (int v = 0; v < p->nvars; ++v) {
    const int c = p->var_cls[(size_t)v];
    const bool gauss = p->cls_kind[(size_t)c] == SPH_FILTER_GAUSS;
    for (int i = 0; i < Nr; ++i) {
      // a pass is the identity where every multiplier is 1: exp and sharp filters with cutoff >= Nyquist
      if (gauss || p->h_lmax[(size_t)c * Nr + i] < (double)Nth) lth.push_back(v * Nr + i);
      for (int j = 0; j < Nth; ++j)
        if (gauss || p->h_mmax[((size_t)c * Nr + i) * Nth + j] < (double)(Nph / 2)) lph.push_back((v * Nr + i) * Nth + j);
    }
    T->pass[0].var_off.push_back((long long)lth.size());
    T->pass[1].var_off.push_back((long long)lph.size());
  }
  // identity theta shells, in runs of consecutive shells per field (copied by out-of-place calls)
  {
    std::vector<char> act((size_t)p->nvars * Nr, 0);
    for (int e : lth) act[(size_t)e] = 1;
    for (int v = 0; v < p->nvars; ++v)
      for (int i = 0; i < Nr;) {
        if (act[(size_t)v * Nr + i]) {
          ++i;
          continue;
        }
        int j = i;
        while (j < Nr && !act[(size_t)v * Nr + j]) ++j;
        T->pass[0].copy_runs.insert(T->pass[0].copy_runs.end(), {v, i, j - i});
        i = j;
      }
  }
  auto up = [](auto** d, const auto& h) -> sph_status {
    if (h.empty()) return SPH_OK;
    if (cudaMalloc((void**)d, h.size() * sizeof(h[0])) != cudaSuccess) return SPH_ENOMEM;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice) == cudaSuccess ? SPH_OK
                                                                                                      : SPH_ECUDA;
  };
  st = up(&T->pass[0].d_h, hth);
  if (st == SPH_OK) st = up(&T->pass[1].d_h, hph);
  if (st == SPH_OK) st = up(&T->pass[0].d_list, lth);
  if (st == SPH_OK) st = up(&T->pass[1].d_list, lph);
  if (st != SPH_OK) return st;
  if (cudaDeviceGetAttribute(&T->nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return SPH_ECUDA;
  const int Hmax = std::max(Lth, Lph) / 2;
  const size_t per_cta = (size_t)tcx::kM * (3 * Hmax + 1);
  T->scratch_set = per_cta * T->nsm;
  if (cudaMalloc((void**)&T->d_scratch, T->scratch_set * sizeof(float2)) != cudaSuccess) return SPH_ENOMEM;
  // kept A stages for GEMMs whose outputs take two passes of the K loop
  for (int q = 0; q < 2; ++q)
    for (int o = 0; o < 4; ++o)
      if (T->pass[q].op[o].nh > 1) T->akeep_chunks = std::max(T->akeep_chunks, T->pass[q].op[o].KP / tcx::kKC);
  T->akeep_set = (size_t)T->akeep_chunks * (tcx::kStageA / 16) * T->nsm;
  if (T->akeep_chunks > 0 && cudaMalloc((void**)&T->d_akeep, T->akeep_set * sizeof(uint4)) != cudaSuccess)
    return SPH_ENOMEM;
  if (cudaFuncSetAttribute(tcx::tc_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcx::kSmemBytes) !=
      cudaSuccess)
    return SPH_ECUDA;
  return SPH_OK;
}

void tc_free(sph_filter_plan_s* p) {
  TcPlan* T = p->tc;
  if (!T) return;
  for (TcPass& P : T->pass) {
    cudaFree(P.d_tab);
    cudaFree(P.d_h);
    cudaFree(P.d_list);
  }
  cudaFree(T->d_scratch);
  cudaFree(T->d_akeep);
  cudaFree(T->d_scratch_pipe);
  cudaFree(T->d_akeep_pipe);
  delete T;
  p->tc = nullptr;
}

sph_status tc_reserve_pipeline(sph_filter_plan_s* p) {
  TcPlan* T = p->tc;
  if (T->d_scratch_pipe) return SPH_OK;
  if (cudaMalloc((void**)&T->d_scratch_pipe, 3 * T->scratch_set * sizeof(float2)) != cudaSuccess) return SPH_ENOMEM;
  if (T->akeep_set && cudaMalloc((void**)&T->d_akeep_pipe, 3 * T->akeep_set * sizeof(uint4)) != cudaSuccess) {
    cudaFree(T->d_scratch_pipe);
    T->d_scratch_pipe = nullptr;
    return SPH_ENOMEM;
  }
  return SPH_OK;
}

namespace {
cudaError_t launch_pass(sph_filter_plan_s* p, int q, const double* src, double* dst, int var_begin, int var_count,
                        cudaStream_t s, int set) {
  TcPlan* T = p->tc;
  TcPass& P = T->pass[q];
  const long long e0 = P.var_off[(size_t)var_begin], e1 = P.var_off[(size_t)(var_begin + var_count)];
  if (e1 <= e0) return cudaSuccess;
  tcx::TcArgs a{};
  a.pass = q;
  a.L = P.L;
  a.Nr = p->Nr;
  a.Nth = p->Nth;
  a.Nph = p->Nph;
  a.src = src;
  a.dst = dst;
  a.list = P.d_list + e0;
  a.nvec = q == 0 ? (e1 - e0) * (p->Nph / 2) : (e1 - e0);
  a.h = P.d_h;
  a.var = p->d_var;
  for (int o = 0; o < 4; ++o) a.op[o] = P.op[o];
  a.Ef = P.Ef;
  a.Ei = P.Ei;
  a.scratch = set == 0 ? T->d_scratch : T->d_scratch_pipe + (size_t)(set - 1) * T->scratch_set;
  a.akeep = set == 0 ? T->d_akeep : (T->d_akeep_pipe ? T->d_akeep_pipe + (size_t)(set - 1) * T->akeep_set : nullptr);
  a.akeep_chunks = T->akeep_chunks;
  a.status = p->d_status;
  const long long ntiles = (a.nvec + tcx::kM - 1) / tcx::kM;
  const int grid = (int)std::min<long long>(ntiles, T->nsm);
  tcx::tc_pass_kernel<<<grid, tcx::kThr, tcx::kSmemBytes, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t tc_launch(sph_filter_plan_s* p, const double* in, double* out, int transpose, int var_begin,
                      int var_count, cudaStream_t s, int set) {
  if (set < 0 || set > 3 || (set > 0 && !p->tc->d_scratch_pipe)) return cudaErrorInvalidValue;
  const size_t shell = (size_t)p->Nth * p->Nph, field = shell * p->Nr;
  if (!transpose) {
    // theta pass in -> out (identity shells copied), then the phi pass in place (Sec. II.C order)
    if (in != out) {
      const std::vector<int>& runs = p->tc->pass[0].copy_runs;
      for (size_t n = 0; n + 2 < runs.size(); n += 3) {
        const int v = runs[n], i0 = runs[n + 1], cnt = runs[n + 2];
        if (v < var_begin || v >= var_begin + var_count) continue;
        const size_t off = field * v + shell * i0;
        const cudaError_t e =
            cudaMemcpyAsync(out + off, in + off, sizeof(double) * shell * cnt, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
      }
    }
    const cudaError_t e = launch_pass(p, 0, in, out, var_begin, var_count, s, set);
    if (e != cudaSuccess) return e;
    return launch_pass(p, 1, out, out, var_begin, var_count, s, set);
  }
  // transpose: phi pass, then theta pass, both in place on out
  if (in != out) {
    const cudaError_t e = cudaMemcpyAsync(out + field * var_begin, in + field * var_begin,
                                          sizeof(double) * field * var_count, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = launch_pass(p, 1, out, out, var_begin, var_count, s, set);
  if (e != cudaSuccess) return e;
  return launch_pass(p, 0, out, out, var_begin, var_count, s, set);
}

}  // namespace sph
