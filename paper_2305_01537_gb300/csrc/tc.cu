// Split-precision tensor-core form of the double FFT filter (SPH_PREC_SPLIT_TC).
//
// Each pass of Sec. II.C applies to every vector c of length L (a doubled great circle, L =
// 2 Ntheta, with the field's parity sign across the pole; or a ring, L = Nphi) the symmetric
// circulant H = F^-1 diag(mu) F that removes the filtered part of each Fourier mode (mu_m = 1 -
// f(|m|, cutoff)), and writes c - H c. Only H c is computed from low-precision products, and the
// subtraction from the field is exact fixed-point arithmetic on 56-bit integers.
//
// One CTA filters 64 vectors of one length at a time (a tile), persistent over the pass's tiles:
//  1. load: the vectors are read from HBM into a shared-memory store of 64-bit fixed-point
//     integers (each vector on its own power-of-two scale);
//  2. symmetry split (tc_plan.cu): in-place sum/difference stages turn each vector into the
//     coordinates of its symmetry blocks; each level's two halves share one operator, so they fill
//     the 128 rows of one GEMM (64 vectors x 2 halves);
//  3. per block GEMM pair: the coordinates of the 128 rows, brought to 46 bits by a per-row shift,
//     are written as six balanced base-256 digits (each exact in BF16) into tensor memory, the A
//     operand of tcgen05.mma (kind::f16); the block's orthonormal mode basis U, as six digit slices,
//     is the B operand, copied to shared memory by the bulk-copy engine. The 21 digit pairs with
//     a + b <= 5 are multiplied; each diagonal a + b = t sums integers of one scale, exactly (< 2^22
//     units) in its own FP32 accumulator (t = 0 .. 3); the two smallest (4 and 5) share one, the
//     diagonal-5 sum scaled by 2^-8 by the MMA's input scaling when diagonal 4 starts. The five
//     accumulators are combined into a 64-bit integer, multiplied by the vector's mu_m (a 62-bit
//     fixed-point fraction), rescaled per row and sliced again as the A operand of the second GEMM
//     (U^T). Its result is subtracted from the stored coordinates;
//  4. the stages are undone in place and the results written back to HBM in FP64.
// Accuracy: every integer step is exact; the errors are the input's rounding to the store (2^-(F+1)
// of the vector's largest value), the dropped digit pairs a + b >= 6 and the truncation to 46 bits
// at the two slicings (about 2^-44 of each row's largest value each), and the rounding of W back to
// the store's unit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "tc2_host.h"

namespace sph {
namespace tcx {

constexpr long long kWaitLimit = 1LL << 24;  // bounded mbarrier polls (about a second at most)
constexpr int kMaxChunks = 3;                // 8-value chunks per thread and row in the mid step

struct RowInfo {
  long long base;                  // offset of the vector's element 0 in the state (circle: meridian k)
  const double* src;               // state the vector is read from
  const uint2* mu;                 // the vector's multipliers mu_m as (mu 2^30, low bits 2^60), m = 0 .. L/2
  int shell;                       // v * Nr + i
  int neg;                         // theta circles of odd fields: the second meridian carries -1
  int valid;
};

// Per pass (0: theta, doubled circles; 1: phi, rings).
struct PassArgs {
  const int* list;                 // theta: active shells v*Nr+i; phi: active rings (v*Nr+i)*Nth+j
  const uint2* mu;                 // theta: [ncls][Nr][Nth+1]; phi: [ncls][Nr][Nth][Nph/2+1]
  const unsigned char* ops;        // operator blob (global), layout of the pass's PassDesc
};

// Work items (int4): {0, first circle, circles, 0} a theta tile; {1, first ring of the list, rings,
// depends} a phi tile (depends: some ring's shell has a theta pass, whose circles must be done
// first); {2, shell, first ring, rings} a copy of rings without any pass (out-of-place calls).
enum { kItemTheta = 0, kItemPhi = 1, kItemCopy = 2 };

struct TcArgs {
  int Nr, Nth, Nph;
  int var_begin, var_end;          // fields [var_begin, var_end) are filtered
  const double* in;
  double* out;                     // may equal in
  int fused;                       // 1: phi tiles of shells with a theta pass read `out` after waiting for
                                   // their circles; 0: every tile reads `in` (one pass per launch)
  const VarInfo* var;
  PassDesc pd[2];
  PassArgs pa[2];
  // direct form (theta pass, tiles inside one shell): per (class, radius) block matrices
  // U^T diag(mu) U; dop_off / dpb [(cls * Nr + i) * ngemm + g]: byte offset in dops, scale bits
  int direct;
  const unsigned char* dops;
  const uint32_t* dop_off;
  const int8_t* dpb;
  const unsigned char* shell_th;   // [nvars * Nr]: the shell has a theta pass
  int* circles;                    // [nvars * Nr]: theta circles done in this application
  int nshells;
  unsigned* status;
};

// Sizes the kernel is launched for (the largest over its passes and grids).
struct KShape {
  int Lmax;
  uint32_t opmax;
  int tmem_cols;
};

// One plan's application.
struct PlanArgs {
  TcArgs a;
  KShape shape;
  const int4* items;
  int nitems;
  int* work;                       // [0] next item, [1] CTAs finished
};

// Several plans' applications in one launch: item.x = type | grid << 4.
constexpr int kMaxGrids = 8;
struct BatchArgs {
  TcArgs g[kMaxGrids];
  int ngrids;
  KShape shape;
  const int4* items;
  int nitems;
  int* work;
};

struct Ctl {
  RowInfo row[kV];
  int vexp[kV];                    // largest biased FP64 exponent of each vector
  int rowbl[kM];                   // bit length of the largest |value| of a GEMM row
  int sh_mid[kM];                  // per-row shift of the mid-step slicing
  unsigned long long op_bar, mma_bar;
  uint32_t tslot;
  int abort;
  int item[2];
  int last;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle (core matrices of 8 rows x
// 16 bytes; next along K 128 bytes on; next 8-row group (K/8) 128 bytes on).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, int K) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(((K / 8) * 128) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128.
__device__ __forceinline__ uint32_t make_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

// Bounded wait on an mbarrier phase (about a second at most).
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

// Bulk copy (TMA engine) of `bytes` (multiple of 16) from global to shared memory, completing on
// the mbarrier; issued by one thread after arming the barrier with the byte count.
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  const char* g = static_cast<const char*>(gsrc);
  uint32_t s = su32(sdst);
  for (uint32_t off = 0; off < bytes; off += 16384) {
    const uint32_t n = bytes - off < 16384 ? bytes - off : 16384;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s + off),
        "l"(g + off), "r"(n), "r"(bar)
        : "memory");
  }
}

// round(x 2^(F - ex)) of the FP64 bit pattern b for |x| < 2^ex, with base = 1075 - F + ex
// (zero and subnormal inputs give 0).
__device__ __forceinline__ long long to_fixed(long long b, int base) {
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int sh = base - e;
  long long t;
  if (sh <= 0) t = m << (-sh);  // -sh <= 3 since |x| < 2^ex and F <= 56
  else if (sh >= 62) t = 0;
  else t = ((m >> (sh - 1)) + 1) >> 1;
  return b < 0 ? -t : t;
}

// v 2^expo as FP64 (round half away from zero on the dropped bits; 0 on underflow).
__device__ __forceinline__ double from_fixed(long long v, int expo) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? 0x8000000000000000ULL : 0ULL;
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long r = (a >> 11) + ((a >> 10) & 1ULL);
  int be = 63 - lz + expo + 1023;
  if (r >> 53) {
    r >>= 1;
    ++be;
  }
  if (be <= 0) return __longlong_as_double((long long)sgn);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (r & 0xFFFFFFFFFFFFFULL)));
}

// The GEMM result from the five accumulators, sum_t acc_t 2^(80 - 8t - Pb), acc 4 holding diagonal 4
// plus diagonal 5 / 256. Each accumulator is an integer below 2^22 (acc 4 rounded to one): adding
// 1.5 2^23 leaves it in the low mantissa bits; m[0..2] = 2^(72 - Pb), 2^(56 - Pb), 2^(48 - Pb).
__device__ __forceinline__ long long combine5(float a0, float a1, float a2, float a3, float a4, const int m[3]) {
  const unsigned b0 = (unsigned)__float_as_int(__fadd_rn(a0, 12582912.0f));
  const unsigned b1 = (unsigned)__float_as_int(__fadd_rn(a1, 12582912.0f));
  const unsigned b2 = (unsigned)__float_as_int(__fadd_rn(a2, 12582912.0f));
  const unsigned b3 = (unsigned)__float_as_int(__fadd_rn(a3, 12582912.0f));
  const unsigned b4 = (unsigned)__float_as_int(__fadd_rn(a4, 12582912.0f));
  const unsigned kM257 = 257u * 0x4B400000u;  // (b - M) 256 + (b' - M) = 256 b + b' - 257 M (mod 2^32)
  const int hi = (int)(b0 * 256u + b1 - kM257);
  const int lo = (int)(b2 * 256u + b3 - kM257);
  const int i4 = (int)(b4 - 0x4B400000u);
  return (long long)hi * m[0] + (long long)lo * m[1] + (long long)i4 * m[2];
}

// d mu for mu = mh 2^-30 + ml 2^-60 (mh <= 2^30, ml < 2^30), with 32-bit limbs of d; the dropped
// low-by-low product is below 4 units of d.
__device__ __forceinline__ long long mul_mu(long long d, uint2 mu) {
  const int dh = (int)(d >> 32);
  const unsigned dl = (unsigned)d;
  const long long t1 = (long long)dh * (int)mu.x;                    // 2^2 weight
  const unsigned long long t2 = (unsigned long long)dl * mu.x;       // 2^-30 weight
  const long long t3 = (long long)dh * (int)mu.y;                    // 2^-28 weight
  return (t1 << 2) + (long long)(t2 >> 30) + (t3 >> 28);
}


__device__ __forceinline__ int bitlen(unsigned long long v) { return v ? 64 - __clzll((long long)v) : 0; }

// Digit byte k of x as the float (byte - 128): the float 2^23 + byte built with a byte permute.
__device__ __forceinline__ float digit_f(uint32_t x, int k) {
  return __fsub_rn(__uint_as_float(__byte_perm(x, 0x4B000000u, 0x7540u + (uint32_t)k)), 8388736.0f);
}

// Six BF16 digit slices of eight values (|v| <= 2^46): w[a][i] packs values 2i, 2i + 1 of slice a.
__device__ __forceinline__ void slice8(const long long v[8], uint32_t w[kS][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned long long t0 = (unsigned long long)(v[2 * i] + 0x808080808080LL);
    const unsigned long long t1 = (unsigned long long)(v[2 * i + 1] + 0x808080808080LL);
    const uint32_t l0 = (uint32_t)t0, h0 = (uint32_t)(t0 >> 32), l1 = (uint32_t)t1, h1 = (uint32_t)(t1 >> 32);
    const uint32_t x0[kS] = {h0, h0, l0, l0, l0, l0}, x1[kS] = {h1, h1, l1, l1, l1, l1};
    const int byte[kS] = {1, 0, 3, 2, 1, 0};
#pragma unroll
    for (int a = 0; a < kS; ++a) {
      const __nv_bfloat162 p = __floats2bfloat162_rn(digit_f(x0[a], byte[a]), digit_f(x1[a], byte[a]));
      w[a][i] = *reinterpret_cast<const uint32_t*>(&p);
    }
  }
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t w[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3])
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float f[8]) {
  uint32_t v[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) f[i] = __uint_as_float(v[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

struct Kern {
  const TcArgs* A;           // the current item's grid
  const PassDesc* d;         // the current tile's pass
  int pass;
  Ctl& C;
  unsigned char* opbuf;      // operator buffer (shared)
  long long* store;          // [kV][pitch] fixed-point store
  int pitch;
  uint32_t tmem;
  int tid, warp, lane, lq, cp, WQ, r, h, v;   // thread role in the GEMM phases: row r = 32 lq + lane
  uint32_t op_phase, mma_phase;
};

// One tcgen05.mma (kind::f16, A in tensor memory, B in shared memory): D = A B^T (+ D) or, with the
// input scaling, D = A B^T + D 2^-8.
__device__ __forceinline__ void mma_first(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 0, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
               "r"(a), "l"(b), "r"(idesc));
}
__device__ __forceinline__ void mma_acc(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
               "r"(a), "l"(b), "r"(idesc));
}
__device__ __forceinline__ void mma_acc_scaled(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p, 8;\n\t}" ::"r"(d),
               "r"(a), "l"(b), "r"(idesc));
}

// Issue the MMAs of one GEMM: D (columns N) = A (tensor memory, K = 16 NKS) x B^T (shared, N x K),
// the 21 digit pairs a + b <= 5 into 5 accumulators (diagonals 5 and 4 first, into accumulator 4,
// the first diagonal-4 product scaling the diagonal-5 sum by 2^-8), then commit to the MMA barrier.
// One thread; every address is a compile-time offset from the bases.
template <int NKS>
__device__ __forceinline__ void issue_gemm_t(uint32_t tmem, uint32_t acc0, int KAh, int NA, uint64_t bd0,
                                             uint32_t slice16, uint32_t idesc) {
#pragma unroll
  for (int t = 5; t >= 0; --t) {
    const uint32_t dcol = acc0 + (uint32_t)((t >= 4 ? 4 : t) * NA);
#pragma unroll
    for (int s = 0; s < NKS; ++s)
#pragma unroll
      for (int a = 0; a <= t; ++a) {
        const int b = t - a;
        const uint32_t acol = tmem + (uint32_t)(a * KAh + s * 8);
        const uint64_t bd = bd0 + (uint64_t)((uint32_t)b * slice16 + (uint32_t)s * 16u);
        if (s == 0 && a == 0 && (t == 5 || t <= 3)) mma_first(dcol, acol, bd, idesc);
        else if (s == 0 && a == 0 && t == 4) mma_acc_scaled(dcol, acol, bd, idesc);
        else mma_acc(dcol, acol, bd, idesc);
      }
  }
}

__device__ void issue_gemm(Kern& k, int K, int N) {
  const PassDesc& d = *k.d;
  const uint32_t idesc = make_idesc(N);
  const uint32_t slice16 = (uint32_t)(N * K * 2) >> 4;
  const uint64_t bd0 = make_desc(su32(k.opbuf), K);
  const uint32_t acc0 = k.tmem + (uint32_t)(3 * d.KA);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  switch (K / 16) {
    case 1: issue_gemm_t<1>(k.tmem, acc0, d.KA / 2, d.NA, bd0, slice16, idesc); break;
    case 2: issue_gemm_t<2>(k.tmem, acc0, d.KA / 2, d.NA, bd0, slice16, idesc); break;
    case 3: issue_gemm_t<3>(k.tmem, acc0, d.KA / 2, d.NA, bd0, slice16, idesc); break;
    default: issue_gemm_t<4>(k.tmem, acc0, d.KA / 2, d.NA, bd0, slice16, idesc); break;
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&k.C.mma_bar))
               : "memory");
}

// Runs one GEMM: a barrier (every thread's A operand and its reads of the previous GEMM's
// accumulators are done), thread 0 waits for the operator, issues and waits for the completion,
// and a second barrier releases the others (who sleep at it instead of polling). A wait that runs
// out sets `abort`.
__device__ void run_gemm(Kern& k, int K, int N) {
  tmem_wait_st();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (k.tid == 0) {
    // the operator copy and the MMAs were issued by this CTA: wait for them even after an abort
    // elsewhere, so that nothing is in flight when the CTA leaves
    if (mbar_wait(su32(&k.C.op_bar), k.op_phase & 1u)) {
      issue_gemm(k, K, N);
      if (!mbar_wait(su32(&k.C.mma_bar), k.mma_phase & 1u)) k.C.abort = 1;
    } else {
      k.C.abort = 1;
    }
  }
  k.op_phase++;
  k.mma_phase++;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Slices 8 values of row r into the A region at K offset k0 (6 slices).
__device__ __forceinline__ void put_a(const Kern& k, const long long vals[8], int k0) {
  uint32_t w[kS][4];
  slice8(vals, w);
  const uint32_t lane_base = k.tmem + ((uint32_t)(32 * k.lq) << 16);
#pragma unroll
  for (int a = 0; a < kS; ++a) tmem_st4(lane_base + (uint32_t)(a * (k.d->KA / 2) + k0 / 2), w[a]);
}

// Prologue: the GEMM's input coordinates of row r, shifted right by the block's bound (|c| < 2^(F +
// growth) becomes |A| < 2^46), as the A operand.
__device__ void prologue(Kern& k, const GemmDesc& g) {
  const int cnt = k.C.row[k.v].valid ? g.cnt[k.h] : 0;
  const long long* srow = k.store + (size_t)k.v * k.pitch + g.ka[k.h];
  const int ks = g.ks[k.h];
  const int nch = g.Kc / 8;
  for (int c = k.cp; c < nch; c += k.WQ) {
    long long vals[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = 8 * c + i;
      vals[i] = kk < cnt ? (srow[ks * kk] >> g.rin) : 0;
    }
    put_a(k, vals, 8 * c);
  }
}

// Mid step: forward GEMM result -> times mu_m -> rescaled per row -> the inverse GEMM's A operand.
__device__ void mid_step(Kern& k, const GemmDesc& g) {
  const int cnt = k.C.row[k.v].valid ? g.cnt[k.h] : 0;
  const uint2* mu = k.C.row[k.v].mu + g.ma[k.h];
  const int ms = g.ms[k.h];
  const int coff = g.concat ? k.h * g.Km : 0;
  const int mlt[3] = {1 << (72 - g.Pb), 1 << (56 - g.Pb), 1 << (48 - g.Pb)};
  const uint32_t lane_base = k.tmem + ((uint32_t)(32 * k.lq) << 16);
  const uint32_t accb = lane_base + (uint32_t)(3 * k.d->KA);
  const int nch = g.Km / 8;
  long long y[kMaxChunks][8];
  unsigned long long orv = 0;
#pragma unroll
  for (int ci = 0; ci < kMaxChunks; ++ci) {
    const int c = k.cp + ci * k.WQ;
    if (c < nch) {
      float f[5][8];
#pragma unroll
      for (int t = 0; t < 5; ++t) tmem_ld8(accb + (uint32_t)(t * k.d->NA + coff + 8 * c), f[t]);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const long long yy =
            8 * c + i < cnt ? mul_mu(combine5(f[0][i], f[1][i], f[2][i], f[3][i], f[4][i], mlt), __ldg(mu + ms * (8 * c + i))) : 0;
        y[ci][i] = yy;
        orv |= (unsigned long long)(yy ^ (yy >> 63));
      }
    }
  }
  if (orv) atomicMax(&k.C.rowbl[k.r], bitlen(orv));
  __syncthreads();
  // |Y| brought to 46 bits, but never scaled up by more than the prologue's right shift, so that
  // the epilogue's shift back to the store's unit is a left shift
  const int bl = k.C.rowbl[k.r];
  const int sm = min(g.rin, bl ? 46 - bl : g.rin);
#pragma unroll
  for (int ci = 0; ci < kMaxChunks; ++ci) {
    const int c = k.cp + ci * k.WQ;
    if (c < nch) {
      long long vals[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) vals[i] = sm >= 0 ? (y[ci][i] << sm) : (y[ci][i] >> (-sm));
      put_a(k, vals, 8 * c);
    }
  }
  if (k.cp == 0) k.C.sh_mid[k.r] = sm;
}

// Epilogue: the inverse GEMM's result W (units 2^(rin - sh_mid) of the store) subtracted from the
// stored coordinates.
__device__ void epilogue(Kern& k, const GemmDesc& g) {
  const int cnt = k.C.row[k.v].valid ? g.cnt[k.h] : 0;
  const int ks = g.ks[k.h];
  const int coff = g.concat ? k.h * g.Kc : 0;
  const uint32_t lane_base = k.tmem + ((uint32_t)(32 * k.lq) << 16);
  const uint32_t accb = lane_base + (uint32_t)(3 * k.d->KA);
  const int mlt[3] = {1 << (72 - g.Pb), 1 << (56 - g.Pb), 1 << (48 - g.Pb)};
  const int up = g.rin - k.C.sh_mid[k.r];  // >= 0
  if (k.cp == 0) k.C.rowbl[k.r] = 0;         // every thread read it before the inverse GEMM's barrier
  long long* srow = k.store + (size_t)k.v * k.pitch + g.ka[k.h];
  const int nch = g.Kc / 8;
  for (int c = k.cp; c < nch; c += k.WQ) {
    float f[5][8];
#pragma unroll
    for (int t = 0; t < 5; ++t) tmem_ld8(accb + (uint32_t)(t * k.d->NA + coff + 8 * c), f[t]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = 8 * c + i;
      if (kk >= cnt) continue;
      const long long w = combine5(f[0][i], f[1][i], f[2][i], f[3][i], f[4][i], mlt);
      srow[ks * kk] -= w << up;
    }
  }
}

// Epilogue of the direct form: the GEMM's result W = K A (units 2^rin of the store) subtracted from
// the stored coordinates.
__device__ void epilogue_direct(Kern& k, const GemmDesc& g, int Pb) {
  const int cnt = k.C.row[k.v].valid ? g.cnt[k.h] : 0;
  const int ks = g.ks[k.h];
  const int coff = g.concat ? k.h * g.Kc : 0;
  const uint32_t lane_base = k.tmem + ((uint32_t)(32 * k.lq) << 16);
  const uint32_t accb = lane_base + (uint32_t)(3 * k.d->KA);
  const int mlt[3] = {1 << (72 - Pb), 1 << (56 - Pb), 1 << (48 - Pb)};
  long long* srow = k.store + (size_t)k.v * k.pitch + g.ka[k.h];
  const int nch = g.Kc / 8;
  for (int c = k.cp; c < nch; c += k.WQ) {
    float f[5][8];
#pragma unroll
    for (int t = 0; t < 5; ++t) tmem_ld8(accb + (uint32_t)(t * k.d->NA + coff + 8 * c), f[t]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = 8 * c + i;
      if (kk >= cnt) continue;
      const long long w = combine5(f[0][i], f[1][i], f[2][i], f[3][i], f[4][i], mlt);
      srow[ks * kk] -= w << g.rin;
    }
  }
}

// Runs f(st, p) for every vector v of the tile and p < count, st = init(v) computed once per vector
// a thread visits, without divisions: theta circles take the vector from the thread (consecutive
// threads, consecutive circles: coalesced meridian rows), rings one warp per vector (consecutive
// lanes, consecutive positions).
template <class Init, class Fn>
__device__ __forceinline__ void for_vec(const Kern& k, int count, Init init, Fn f) {
  if (k.pass == 0) {
    const auto st = init(k.tid & (kV - 1));
    for (int p = k.tid >> 6; p < count; p += (int)(blockDim.x >> 6)) f(st, p);
  } else {
    for (int v = k.warp; v < kV; v += (int)(blockDim.x >> 5)) {
      const auto st = init(v);
      for (int p = k.lane; p < count; p += 32) f(st, p);
    }
  }
}

// A vector's store row and the conversion of its raw FP64 values: base = 53 - F + its exponent; on
// a theta circle the second meridian carries the field's parity sign (neg).
struct VecIn {
  long long* s;
  int base;
  bool neg;
};
__device__ __forceinline__ VecIn vec_in(const Kern& k, int v) {
  return VecIn{k.store + (size_t)v * k.pitch, 53 - k.d->F + k.C.vexp[v], k.pass == 0 && k.C.row[v].neg != 0};
}

// In-place level stage (forward) on the first n entries of every vector's store.
__device__ void level_fwd(Kern& k, int n, bool convert) {
  const int q = n / 4;
  for_vec(k, q, [&](int v) { return vec_in(k, v); }, [&](const VecIn& V, int p) {
    long long* s = V.s;
    long long vp = s[p], vq = s[p + n / 2], vr = s[n / 2 - 1 - p], vs = s[n - 1 - p];
    if (convert) {
      // the outermost level reads the raw FP64 values; on a theta circle positions p + n/2 and
      // n - 1 - p lie on the second meridian
      vp = to_fixed(vp, V.base);
      vq = to_fixed(vq, V.base);
      vr = to_fixed(vr, V.base);
      vs = to_fixed(vs, V.base);
      if (V.neg) {
        vq = -vq;
        vs = -vs;
      }
    }
    const long long e0 = vp + vq, z0 = vp - vq, e1 = vr + vs, z1 = vr - vs;
    s[p] = e0;
    s[n / 2 - 1 - p] = e1;
    s[n / 2 + p] = z0 - z1;
    s[n - 1 - p] = z0 + z1;
  });
}

__device__ void base_fwd(Kern& k, int nb, bool convert) {
  for_vec(k, nb / 2, [&](int v) { return vec_in(k, v); }, [&](const VecIn& V, int p) {
    long long* s = V.s;
    long long a = s[p], b = s[nb - 1 - p];
    if (convert) {
      // no levels: nb = L; on a theta circle position nb - 1 - p is on the second meridian
      a = to_fixed(a, V.base);
      b = to_fixed(b, V.base);
      if (V.neg) b = -b;
    }
    s[p] = a + b;
    s[nb - 1 - p] = a - b;
  });
}

// A vector's store row and its destination: position q of a theta circle is at top + q Nphi on the
// first meridian (q < Ntheta) and at bot - q Nphi on the second, with the parity sign applied to
// the integer; a ring's position q is at top + q. Values are scaled by 2^expo.
struct VecOut {
  long long* s;
  double* top;
  double* bot;
  int expo, nth, nph;
  bool neg, valid;
};
__device__ __forceinline__ VecOut vec_out(const Kern& k, int v, int shift) {
  const RowInfo& R = k.C.row[v];
  const int nth = k.A->Nth, nph = k.A->Nph;
  double* top = k.A->out + R.base;
  return VecOut{k.store + (size_t)v * k.pitch, top, top + (long long)(2 * nth - 1) * nph + nph / 2,
                (k.C.vexp[v] - 1022) - k.d->F - shift, nth, nph, k.pass == 0 && R.neg != 0, R.valid != 0};
}
__device__ __forceinline__ void put_out(const Kern& k, const VecOut& V, int q, long long x) {
  double* dst;
  if (k.pass == 0) {
    const bool up = q < V.nth;
    if (V.neg && !up) x = -x;
    dst = up ? V.top + (long long)q * V.nph : V.bot - (long long)q * V.nph;
  } else {
    dst = V.top + q;
  }
  *dst = from_fixed(x, V.expo);
}

// Inverse base stage: values become 2 v; `out` writes them to the destination (no levels).
__device__ void base_inv(Kern& k, int nb, bool out) {
  if (out) {
    for_vec(k, nb / 2, [&](int v) { return vec_out(k, v, 1); }, [&](const VecOut& V, int p) {
      if (!V.valid) return;
      const long long a = V.s[p], b = V.s[nb - 1 - p];
      put_out(k, V, p, a + b);
      put_out(k, V, nb - 1 - p, a - b);
    });
    return;
  }
  for_vec(k, nb / 2, [&](int v) { return k.store + (size_t)v * k.pitch; }, [&](long long* s, int p) {
    const long long a = s[p], b = s[nb - 1 - p];
    s[p] = a + b;
    s[nb - 1 - p] = a - b;
  });
}

// Inverse level stage for the level of length n, with the T-even part scaled by 2^sc (sc >= 1);
// results scaled by 2^(sc + 1). `out` writes them to the destination (outermost level).
__device__ void level_inv(Kern& k, int n, int sc, bool out) {
  auto butterfly = [&](const long long* s, int p, long long y[4]) {
    const long long E0 = s[p], E1 = s[n / 2 - 1 - p], a = s[n / 2 + p], o = s[n - 1 - p];
    const long long zp = (o + a) << (sc - 1), zq = (o - a) << (sc - 1);
    y[0] = E0 + zp;
    y[1] = E0 - zp;
    y[2] = E1 + zq;
    y[3] = E1 - zq;
  };
  if (out) {
    for_vec(k, n / 4, [&](int v) { return vec_out(k, v, sc + 1); }, [&](const VecOut& V, int p) {
      if (!V.valid) return;
      long long y[4];
      butterfly(V.s, p, y);
      put_out(k, V, p, y[0]);
      put_out(k, V, p + n / 2, y[1]);
      put_out(k, V, n / 2 - 1 - p, y[2]);
      put_out(k, V, n - 1 - p, y[3]);
    });
    return;
  }
  for_vec(k, n / 4, [&](int v) { return k.store + (size_t)v * k.pitch; }, [&](long long* s, int p) {
    long long y[4];
    butterfly(s, p, y);
    s[p] = y[0];
    s[p + n / 2] = y[1];
    s[n / 2 - 1 - p] = y[2];
    s[n - 1 - p] = y[3];
  });
}

// Bounded wait (on the GPU, about a second) for a shell's theta circles; false if it ran out.
__device__ __forceinline__ bool wait_circles(const int* ctr, int need) {
  for (long long it = 0; it < (1LL << 22); ++it) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= need) return true;
    __nanosleep(256);
  }
  return false;
}

// Copies rings [j0, j0 + nj) of one shell from in to out (rings no pass changes).
__device__ void copy_rings(const TcArgs& A, int shell, int j0, int nj) {
  const size_t off = ((size_t)shell * A.Nth + j0) * A.Nph;
  const size_t n16 = (size_t)nj * A.Nph / 2;  // 16-byte pieces (Nphi is even)
  const double2* s = reinterpret_cast<const double2*>(A.in + off);
  double2* d = reinterpret_cast<double2*>(A.out + off);
  size_t i = threadIdx.x;
  for (; i + 3 * blockDim.x < n16; i += 4 * blockDim.x) {
    const double2 a = __ldcs(s + i), b = __ldcs(s + i + blockDim.x), c = __ldcs(s + i + 2 * blockDim.x),
                  e = __ldcs(s + i + 3 * blockDim.x);
    __stcs(d + i, a);
    __stcs(d + i + blockDim.x, b);
    __stcs(d + i + 2 * blockDim.x, c);
    __stcs(d + i + 3 * blockDim.x, e);
  }
  for (; i < n16; i += blockDim.x) __stcs(d + i, __ldcs(s + i));
}

// The persistent loop over work items, shared by the one-plan and the several-plan kernels: grids[g]
// holds the arguments of grid g (item.x >> 4 when MULTI, else 0).
template <bool MULTI>
__device__ __forceinline__ void run_items(const TcArgs* grids, int ngrids, const KShape& shape, const int4* items,
                                          int nitems, int* work) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int Lmax = shape.Lmax;
  const uint32_t opmax = shape.opmax;
  const int tmem_cols = shape.tmem_cols;
  unsigned char* opbuf = smem;
  long long* store = reinterpret_cast<long long*>(smem + ((opmax + 1023) / 1024) * 1024);
  Ctl& C = *reinterpret_cast<Ctl*>(store + (size_t)kV * (Lmax + 1));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&C.tslot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&C.op_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&C.mma_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    C.abort = 0;
    C.item[0] = atomicAdd(&work[0], 1);  // the first item
  }
  for (int i = tid; i < kM; i += blockDim.x) C.rowbl[i] = 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  Kern k{grids, &grids[0].pd[0], 0, C, opbuf, store, 0, C.tslot, tid, warp, lane, warp & 3, warp >> 2, (int)(blockDim.x / 128),
         0, 0, 0, 0u, 0u};
  k.r = 32 * k.lq + lane;
  k.h = k.r >> 6;
  k.v = k.r & (kV - 1);
  for (int n = 0;; ++n) {
    // two slots: the item of iteration n + 1 is fetched during iteration n (its atomic's latency
    // hidden behind the tile), into the slot that iteration n - 1 read before the barrier below
    __syncthreads();
    const int it = C.item[n & 1];
    if (it >= nitems || C.abort) break;
    if (tid == 0) C.item[(n + 1) & 1] = atomicAdd(&work[0], 1);
    int4 w = items[it];
    const TcArgs& A = grids[MULTI ? (w.x >> 4) : 0];
    w.x &= 15;
    k.A = &A;
    const int half = A.Nph / 2;
    if (w.x == kItemCopy) {
      const int v = w.y / A.Nr;
      if (A.in != A.out && v >= A.var_begin && v < A.var_end) copy_rings(A, w.y, w.z, w.w);
      continue;  // the barrier at the top of the loop orders the next item
    }
    const int pass = w.x;
    const PassDesc& d = A.pd[pass];
    const PassArgs& P = A.pa[pass];
    k.d = &d;
    k.pass = pass;
    const int L = d.L;
    const int pitch = L + 1;
    k.pitch = pitch;
    // the direct form's operators are those of the tile's (class, radius): every circle of a
    // theta tile lies in one shell
    int dci = 0;
    const bool direct = pass == 0 && A.direct;
    if (direct) {
      const int shell = P.list[w.y / half];
      const int vv = shell / A.Nr, i = shell - vv * A.Nr;
      dci = (A.var[vv].cls * A.Nr + i) * d.ngemm;
    }
    if (tid < kV) {
      RowInfo R{};
      R.valid = 0;
      if (tid < w.z) {
        const long long vg = (long long)w.y + tid;
        int shell, vv, i;
        if (pass == 0) {
          shell = P.list[vg / half];
          vv = shell / A.Nr;
          i = shell - vv * A.Nr;
          R.base = (long long)shell * A.Nth * A.Nph + (int)(vg % half);
          R.mu = P.mu + ((size_t)A.var[vv].cls * A.Nr + i) * (A.Nth + 1);
          R.neg = A.var[vv].parity;
          R.src = A.in;
        } else {
          const int ring = P.list[vg];
          const int j = ring % A.Nth;
          shell = ring / A.Nth;
          vv = shell / A.Nr;
          i = shell - vv * A.Nr;
          R.base = (long long)ring * A.Nph;
          R.mu = P.mu + (((size_t)A.var[vv].cls * A.Nr + i) * A.Nth + j) * (A.Nph / 2 + 1);
          R.neg = 0;
          // in the fused application a shell with a theta pass is read back from out once all its
          // circles are done
          const bool after_theta = A.fused && A.shell_th[shell];
          R.src = after_theta ? A.out : A.in;
          if (after_theta && vv >= A.var_begin && vv < A.var_end &&
              !wait_circles(A.circles + shell, half))
            C.abort = 1;
        }
        R.shell = shell;
        R.valid = vv >= A.var_begin && vv < A.var_end;
      }
      C.row[tid] = R;
      C.vexp[tid] = 0;
    }
    const int any = __syncthreads_or(tid < kV && C.row[tid].valid);
    if (C.abort) break;
    if (!any) continue;  // every vector belongs to fields outside the call's range
    // the first operator (the buffer is free: the previous tile's GEMMs completed)
    if (tid == 0) {
      if (direct) bulk_load(opbuf, A.dops + A.dop_off[dci], d.g[0].Kc * (d.g[0].concat ? 2 : 1) * d.g[0].Kc * 2 * kS, su32(&C.op_bar));
      else bulk_load(opbuf, P.ops + d.g[0].fwd_off, d.g[0].fwd_bytes, su32(&C.op_bar));
    }
    // load: raw FP64 values by asynchronous 8-byte copies (all of a thread's copies in flight at once),
    // then each vector's exponent. A ring read back after its shell's theta tiles cannot be stale in
    // this SM's L1: the only earlier reads of those lines in this launch are by the theta tile that
    // wrote them (and this SM's own writes keep its L1 current)
    {
      struct Src {
        const double* top;
        const double* bot;
        uint32_t dst;
        bool valid;
      };
      const int Nth = A.Nth, Nph = A.Nph;
      for_vec(k, L,
              [&](int v) {
                const RowInfo& R = C.row[v];
                const double* top = R.src + R.base;
                return Src{top, top + (long long)(2 * Nth - 1) * Nph + Nph / 2, su32(store + (size_t)v * pitch),
                           R.valid != 0};
              },
              [&](const Src& S, int q) {
                if (!S.valid) return;
                const double* g = pass != 0 ? S.top + q : (q < Nth ? S.top + (long long)q * Nph : S.bot - (long long)q * Nph);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(S.dst + 8u * (uint32_t)q), "l"(g) : "memory");
              });
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    if (pass == 0) {
      int e = 0;
      const int v = tid & (kV - 1);
      if (C.row[v].valid) {
        const long long* s = store + (size_t)v * pitch;
        for (int q = tid >> 6; q < L; q += (int)(blockDim.x >> 6)) e = max(e, (int)((s[q] >> 52) & 0x7FF));
      }
      atomicMax(&C.vexp[v], e);
    } else {
      for (int v = warp; v < kV; v += blockDim.x / 32) {
        int e = 0;
        if (C.row[v].valid)
          for (int q = lane; q < L; q += 32) e = max(e, (int)((store[(size_t)v * pitch + q] >> 52) & 0x7FF));
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0) C.vexp[v] = e;
      }
    }
    __syncthreads();
    // symmetry split, in place (the first stage converts to fixed point)
    {
      int n = L;
      for (int l = 0; l < d.nl; ++l, n /= 2) {
        level_fwd(k, n, l == 0);
        __syncthreads();
      }
      base_fwd(k, d.nb, d.nl == 0);
      __syncthreads();
    }
    // block GEMMs: the direct form, one per block
    for (int gi = 0; gi < d.ngemm && direct; ++gi) {
      const GemmDesc& g = d.g[gi];
      const int N = g.concat ? 2 * g.Kc : g.Kc;
      prologue(k, g);
      run_gemm(k, g.Kc, N);
      if (tid == 0 && gi + 1 < d.ngemm) {
        const GemmDesc& g2 = d.g[gi + 1];
        bulk_load(opbuf, A.dops + A.dop_off[dci + gi + 1], g2.Kc * (g2.concat ? 2 : 1) * g2.Kc * 2 * kS, su32(&C.op_bar));
      }
      epilogue_direct(k, g, A.dpb[dci + gi]);
    }
    // block GEMM pairs of the factored form
    for (int gi = 0; gi < d.ngemm && !direct; ++gi) {
      const GemmDesc& g = d.g[gi];
      prologue(k, g);
      run_gemm(k, g.Kc, g.concat ? 2 * g.Km : g.Km);
      if (tid == 0) bulk_load(opbuf, P.ops + g.inv_off, g.inv_bytes, su32(&C.op_bar));
      mid_step(k, g);
      run_gemm(k, g.Km, g.concat ? 2 * g.Kc : g.Kc);
      if (tid == 0 && gi + 1 < d.ngemm) bulk_load(opbuf, P.ops + d.g[gi + 1].fwd_off, d.g[gi + 1].fwd_bytes, su32(&C.op_bar));
      epilogue(k, g);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (C.abort) break;
    // undo the split and write the results (FP64)
    if (d.nl == 0) {
      base_inv(k, d.nb, true);
    } else {
      base_inv(k, d.nb, false);
      __syncthreads();
      int sc = 1;
      int n = d.nb * 2;
      for (int l = d.nl - 1; l >= 1; --l, n *= 2, ++sc) {
        level_inv(k, n, sc, false);
        __syncthreads();
      }
      level_inv(k, n, sc, true);
    }
    // a theta tile's circles are done: publish them (every thread's writes first)
    if (pass == 0) {
      __threadfence();
      __syncthreads();
      if (tid < kV && C.row[tid].valid) atomicAdd(A.circles + C.row[tid].shell, 1);
    }
  }
  if (C.abort && tid == 0)
    for (int g = 0; g < ngrids; ++g) atomicCAS(grids[g].status, 0u, (unsigned)SPH_ETIMEOUT);
  // the last CTA to finish resets the counters for the next application
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    C.last = atomicAdd(work + 1, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (C.last) {
    for (int g = 0; g < ngrids; ++g)
      for (int i = tid; i < grids[g].nshells; i += blockDim.x) grids[g].circles[i] = 0;
    if (tid == 0) work[0] = 0;
    __threadfence();
    __syncthreads();
    if (tid == 0) work[1] = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(C.tslot), "r"(tmem_cols));
}

__global__ void __launch_bounds__(512, 1) tc_pass_kernel(const __grid_constant__ PlanArgs P) {
  run_items<false>(&P.a, 1, P.shape, P.items, P.nitems, P.work);
}

__global__ void __launch_bounds__(512, 1) tc_batch_kernel(const __grid_constant__ BatchArgs B) {
  run_items<true>(B.g, B.ngrids, B.shape, B.items, B.nitems, B.work);
}

size_t smem_bytes(const PassDesc& d) {
  const size_t op = (d.op_max + 1023) / 1024 * 1024;
  const size_t store = (size_t)kV * (d.L + 1) * 8;
  return op + store + sizeof(Ctl);
}

}  // namespace tcx

// ---------------------------------------------------------------- host side

struct TcPass {
  tcx::PassDesc d{};
  std::vector<int> h_list;         // the pass's list (host copy)
  std::vector<tcx::GemmBasis> basis;
  unsigned char* d_ops = nullptr;
  // direct form (theta pass when every tile lies inside one shell)
  bool direct = false;
  unsigned char* d_dops = nullptr;
  uint32_t* d_dop_off = nullptr;
  int8_t* d_dpb = nullptr;
  uint2* d_mu = nullptr;
  int* d_list = nullptr;
  std::vector<long long> var_off;  // list entries of fields [0, v): prefix counts
  std::vector<int> copy_runs;      // theta pass: [field, first shell, shells] runs of identity shells
  size_t smem = 0;
  int ctas_per_sm = 1;
};

// Work lists and the per-application counters. Each call takes the next of kSets counter sets; a call
// on a stream waits for the previous user of its set (an event), so calls on different streams can
// overlap. The kernel's last CTA resets its set, so no call needs a memset.
constexpr int kSets = 4;
struct TcPlan {
  TcPass pass[2];
  int nsm = 0;
  int threads = 0, ctas_per_sm = 1;
  size_t smem = 0;
  tcx::KShape shape{};
  int4* d_items = nullptr;          // [fused application | theta tiles | phi tiles], all fields
  int n_fused = 0, n_theta = 0, n_phi = 0;
  std::vector<int4> h_items;        // the same on the host (filtered for calls on a field range)
  // lists of the items that touch a field range [first, first + count), made on first use
  struct RangeItems {
    int4* d = nullptr;
    int n_fused = 0, n_theta = 0, n_phi = 0;
  };
  std::map<std::pair<int, int>, RangeItems> ranges;
  unsigned char* d_shell_th = nullptr;
  int* d_counters = nullptr;        // kSets x (2 + nshells)
  int nshells = 0;
  cudaEvent_t set_ev[kSets] = {};
  bool set_used[kSets] = {};
  unsigned next_set = 0;
  std::mutex mu;
};

namespace {

// mu = x 2^-30 + y 2^-60 with integers x <= 2^30, y < 2^30 (mu in [0, 1], rounded at 2^-60).
uint2 mu_fixed(long double mu) {
  if (mu <= 0) return make_uint2(0u, 0u);
  if (mu >= 1) return make_uint2(1u << 30, 0u);
  const unsigned long long t = (unsigned long long)llroundl(ldexpl(mu, 60));
  return make_uint2((unsigned)(t >> 30), (unsigned)(t & ((1ULL << 30) - 1)));
}

sph_status build_tc_pass(TcPass* P, int L, int device) {
  std::vector<uint16_t> ops;
  std::vector<int16_t> maps;
  if (!tcx::build_pass_desc(L, &P->d, &ops, &maps, &P->basis)) return SPH_EUNSUPPORTED;
  if (cudaMalloc((void**)&P->d_ops, ops.size() * 2) != cudaSuccess) return SPH_ENOMEM;
  if (cudaMemcpy(P->d_ops, ops.data(), ops.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return SPH_ECUDA;
  P->smem = tcx::smem_bytes(P->d);
  const int optin = max_smem_optin(device);
  if ((int)P->smem > optin) return SPH_EUNSUPPORTED;
  P->ctas_per_sm = (P->d.tmem_cols <= 256 && P->d.threads <= 256 && 2 * (P->smem + 1024) <= (size_t)optin) ? 2 : 1;
  // ask for enough shared memory that no SM holds more CTAs than its tensor memory serves at once
  // (a further CTA would wait in tcgen05.alloc until one of them has finished all its tiles)
  P->smem = std::max(P->smem, (size_t)optin / (P->ctas_per_sm + 1) + 1024);
  P->smem = std::min(P->smem, (size_t)optin);
  return SPH_OK;
}

}  // namespace

sph_status tc_setup(sph_filter_plan_s* p) {
  const int Lth = 2 * p->Nth, Lph = p->Nph;
  TcPlan* T = new (std::nothrow) TcPlan();
  if (!T) return SPH_ENOMEM;
  p->tc = T;
  sph_status st = build_tc_pass(&T->pass[0], Lth, p->device);
  if (st == SPH_OK) st = build_tc_pass(&T->pass[1], Lph, p->device);
  if (st != SPH_OK) return st;
  const int Nr = p->Nr, Nth = p->Nth, Nph = p->Nph, ncls = p->ncls;
  // removed fractions mu = 1 - f (Sec. II.C filter functions) as 62-bit fixed-point fractions
  std::vector<uint2> mth((size_t)ncls * Nr * (Nth + 1)), mph((size_t)ncls * Nr * Nth * (Nph / 2 + 1));
  for (int c = 0; c < ncls; ++c)
    for (int i = 0; i < Nr; ++i) {
      const long double lm = p->h_lmax[(size_t)c * Nr + i];
      for (int l = 0; l <= Nth; ++l)
        mth[((size_t)c * Nr + i) * (Nth + 1) + l] = mu_fixed(1.0L - filter_value(p->cls_kind[(size_t)c], l, lm));
      for (int j = 0; j < Nth; ++j) {
        const long double mm = p->h_mmax[((size_t)c * Nr + i) * Nth + j];
        for (int m = 0; m <= Nph / 2; ++m)
          mph[(((size_t)c * Nr + i) * Nth + j) * (Nph / 2 + 1) + m] =
              mu_fixed(1.0L - filter_value(p->cls_kind[(size_t)c], m, mm));
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
  // direct theta operators, per active (class, radius): possible when a tile of 64 doubled circles
  // never spans two shells
  std::vector<unsigned char> dops;
  std::vector<uint32_t> dop_off;
  std::vector<int8_t> dpb;
  TcPass& P0 = T->pass[0];
  P0.direct = (Nph / 2) % tcx::kV == 0;
  if (P0.direct) {
    const int ng = P0.d.ngemm;
    dop_off.assign((size_t)ncls * Nr * ng, 0u);
    dpb.assign((size_t)ncls * Nr * ng, (int8_t)48);
    std::vector<char> need((size_t)ncls * Nr, 0);
    for (int e : lth) {
      const int v = e / Nr, i = e % Nr;
      need[(size_t)p->var_cls[(size_t)v] * Nr + i] = 1;
    }
    std::vector<uint16_t> blob;
    std::vector<long double> mu((size_t)Nth + 1);
    for (int c = 0; c < ncls; ++c)
      for (int i = 0; i < Nr; ++i) {
        if (!need[(size_t)c * Nr + i]) continue;
        const long double lm = p->h_lmax[(size_t)c * Nr + i];
        for (int l = 0; l <= Nth; ++l) mu[(size_t)l] = 1.0L - filter_value(p->cls_kind[(size_t)c], l, lm);
        for (int g = 0; g < ng; ++g) {
          int pb = 48;
          dop_off[((size_t)c * Nr + i) * ng + g] = tcx::append_direct_op(P0.d, g, P0.basis[(size_t)g], mu.data(), &blob, &pb);
          dpb[((size_t)c * Nr + i) * ng + g] = (int8_t)pb;
        }
      }
    dops.resize(blob.size() * 2);
    std::memcpy(dops.data(), blob.data(), dops.size());
  }
  auto up = [](auto** d, const auto& h) -> sph_status {
    if (h.empty()) return SPH_OK;
    if (cudaMalloc((void**)d, h.size() * sizeof(h[0])) != cudaSuccess) return SPH_ENOMEM;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice) == cudaSuccess ? SPH_OK
                                                                                                      : SPH_ECUDA;
  };
  T->pass[0].h_list = lth;
  T->pass[1].h_list = lph;
  st = up(&T->pass[0].d_mu, mth);
  if (st == SPH_OK) st = up(&T->pass[1].d_mu, mph);
  if (st == SPH_OK) st = up(&T->pass[0].d_list, lth);
  if (st == SPH_OK) st = up(&T->pass[1].d_list, lph);
  if (st == SPH_OK) st = up(&P0.d_dops, dops);
  if (st == SPH_OK) st = up(&P0.d_dop_off, dop_off);
  if (st == SPH_OK) st = up(&P0.d_dpb, dpb);
  if (st != SPH_OK) return st;
  if (cudaDeviceGetAttribute(&T->nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return SPH_ECUDA;
  // work lists. Fused application: theta tiles first, then phi tiles and copies that need no theta
  // result, then phi tiles of shells with a theta pass (every theta tile has been taken by then, so
  // their waits are short and cannot block a running tile).
  const int half = Nph / 2;
  const int nshells = p->nvars * Nr;
  std::vector<unsigned char> shell_th((size_t)nshells, 0);
  for (int e : lth) shell_th[(size_t)e] = 1;
  std::vector<int4> th_items, ph_indep, ph_dep, copies;
  const long long ncirc = (long long)lth.size() * half;
  for (long long s = 0; s < ncirc; s += tcx::kV)
    th_items.push_back(make_int4(tcx::kItemTheta, (int)s, (int)std::min<long long>(tcx::kV, ncirc - s), 0));
  for (size_t s = 0; s < lph.size(); s += tcx::kV) {
    const int cnt = (int)std::min<size_t>(tcx::kV, lph.size() - s);
    int dep = 0;
    for (int r = 0; r < cnt; ++r) dep |= shell_th[(size_t)(lph[s + (size_t)r] / Nth)];
    (dep ? ph_dep : ph_indep).push_back(make_int4(tcx::kItemPhi, (int)s, cnt, dep));
  }
  // rings of shells without a theta pass that the phi pass leaves alone: runs of consecutive rings
  {
    std::vector<char> ring_act((size_t)nshells * Nth, 0);
    for (int e : lph) ring_act[(size_t)e] = 1;
    for (int sh = 0; sh < nshells; ++sh) {
      if (shell_th[(size_t)sh]) continue;
      for (int j = 0; j < Nth;) {
        if (ring_act[(size_t)sh * Nth + j]) {
          ++j;
          continue;
        }
        int j1 = j;
        while (j1 < Nth && !ring_act[(size_t)sh * Nth + j1]) ++j1;
        copies.push_back(make_int4(tcx::kItemCopy, sh, j, j1 - j));
        j = j1;
      }
    }
  }
  std::vector<int4> items;
  items.insert(items.end(), th_items.begin(), th_items.end());
  // interleave the independent phi tiles with the copies (compute next to memory-bound work)
  {
    size_t a = 0, b = 0;
    while (a < ph_indep.size() || b < copies.size()) {
      if (a < ph_indep.size()) items.push_back(ph_indep[a++]);
      if (b < copies.size()) items.push_back(copies[b++]);
    }
  }
  items.insert(items.end(), ph_dep.begin(), ph_dep.end());
  T->n_fused = (int)items.size();
  items.insert(items.end(), th_items.begin(), th_items.end());
  T->n_theta = (int)th_items.size();
  items.insert(items.end(), ph_indep.begin(), ph_indep.end());
  items.insert(items.end(), ph_dep.begin(), ph_dep.end());
  T->n_phi = (int)(ph_indep.size() + ph_dep.size());
  T->nshells = nshells;
  T->h_items = items;
  st = up(&T->d_items, items);
  if (st == SPH_OK) st = up(&T->d_shell_th, shell_th);
  if (st != SPH_OK) return st;
  if (cudaMalloc((void**)&T->d_counters, sizeof(int) * kSets * (2 + (size_t)nshells)) != cudaSuccess) return SPH_ENOMEM;
  if (cudaMemset(T->d_counters, 0, sizeof(int) * kSets * (2 + (size_t)nshells)) != cudaSuccess) return SPH_ECUDA;
  for (cudaEvent_t& e : T->set_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SPH_ECUDA;
  // one kernel serves both passes: the larger of the two shapes
  T->threads = std::max(T->pass[0].d.threads, T->pass[1].d.threads);
  const size_t op = std::max(T->pass[0].d.op_max, T->pass[1].d.op_max);
  const int Lmax = std::max(T->pass[0].d.L, T->pass[1].d.L);
  const int tmem = std::max(T->pass[0].d.tmem_cols, T->pass[1].d.tmem_cols);
  T->shape = tcx::KShape{Lmax, (uint32_t)op, tmem};
  T->smem = (op + 1023) / 1024 * 1024 + (size_t)tcx::kV * (Lmax + 1) * 8 + sizeof(tcx::Ctl);
  const int optin = max_smem_optin(p->device);
  if ((int)T->smem > optin) return SPH_EUNSUPPORTED;
  T->ctas_per_sm = (tmem <= 256 && T->threads <= 256 && 2 * (T->smem + 1024) <= (size_t)optin) ? 2 : 1;
  // enough shared memory that no SM holds more CTAs than its tensor memory serves at once (a further
  // CTA would wait in tcgen05.alloc)
  T->smem = std::min(std::max(T->smem, (size_t)optin / (T->ctas_per_sm + 1) + 1024), (size_t)optin);
  if (cudaFuncSetAttribute(tcx::tc_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T->smem) != cudaSuccess)
    return SPH_ECUDA;
  return SPH_OK;
}

void tc_free(sph_filter_plan_s* p) {
  TcPlan* T = p->tc;
  if (!T) return;
  for (TcPass& P : T->pass) {
    cudaFree(P.d_ops);
    cudaFree(P.d_mu);
    cudaFree(P.d_list);
    cudaFree(P.d_dops);
    cudaFree(P.d_dop_off);
    cudaFree(P.d_dpb);
  }
  cudaFree(T->d_items);
  for (auto& kv : T->ranges) cudaFree(kv.second.d);
  cudaFree(T->d_shell_th);
  cudaFree(T->d_counters);
  for (cudaEvent_t e : T->set_ev)
    if (e) cudaEventDestroy(e);
  delete T;
  p->tc = nullptr;
}

// The form keeps no scratch outside the kernel's shared and tensor memory: nothing to reserve.
sph_status tc_reserve_pipeline(sph_filter_plan_s*) { return SPH_OK; }

namespace {
// The kernel arguments of one plan's application (the work and circle counters are set by the caller).
tcx::TcArgs plan_args(sph_filter_plan_s* p, int fused, const double* in, double* out, int var_begin, int var_count) {
  TcPlan* T = p->tc;
  tcx::TcArgs a{};
  a.Nr = p->Nr;
  a.Nth = p->Nth;
  a.Nph = p->Nph;
  a.var_begin = var_begin;
  a.var_end = var_begin + var_count;
  a.in = in;
  a.out = out;
  a.fused = fused;
  a.var = p->d_var;
  for (int q = 0; q < 2; ++q) {
    a.pd[q] = T->pass[q].d;
    a.pa[q].list = T->pass[q].d_list;
    a.pa[q].mu = T->pass[q].d_mu;
    a.pa[q].ops = T->pass[q].d_ops;
  }
  a.direct = T->pass[0].direct ? 1 : 0;
  a.dops = T->pass[0].d_dops;
  a.dop_off = T->pass[0].d_dop_off;
  a.dpb = T->pass[0].d_dpb;
  a.shell_th = T->d_shell_th;
  a.nshells = T->nshells;
  a.status = p->d_status;
  return a;
}

// One launch over the work items [first, first + count): the fused application (fused = 1) or one
// pass (fused = 0), fields [var_begin, var_begin + var_count).
cudaError_t launch_items(sph_filter_plan_s* p, const int4* items, int count, int fused, const double* in, double* out,
                         int var_begin, int var_count, cudaStream_t s, int* nlaunch) {
  TcPlan* T = p->tc;
  if (count <= 0) return cudaSuccess;
  tcx::TcArgs a = plan_args(p, fused, in, out, var_begin, var_count);
  tcx::PlanArgs pa{};
  pa.items = items;
  pa.nitems = count;
  pa.shape = T->shape;
  // a counter set, after its previous user (except inside a graph capture, which orders its own work)
  std::lock_guard<std::mutex> lock(T->mu);
  const int set = (int)(T->next_set++ % kSets);
  pa.work = T->d_counters + (size_t)set * (2 + T->nshells);
  a.circles = pa.work + 2;
  pa.a = a;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  const bool chain = cap == cudaStreamCaptureStatusNone;
  if (chain && T->set_used[set]) {
    e = cudaStreamWaitEvent(s, T->set_ev[set], 0);
    if (e != cudaSuccess) return e;
  }
  const int grid = std::min(count, T->nsm * T->ctas_per_sm);
  tcx::tc_pass_kernel<<<grid, T->threads, T->smem, s>>>(pa);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  if (chain) {
    e = cudaEventRecord(T->set_ev[set], s);
    T->set_used[set] = e == cudaSuccess;
  }
  return e;
}
}  // namespace

// The field of an item (of its first vector for a tile; tiles of consecutive vectors may cover two).
namespace {
void item_fields(const sph_filter_plan_s* p, const int4& w, int* f0, int* f1) {
  const TcPlan* T = p->tc;
  if (w.x == tcx::kItemCopy) {
    *f0 = *f1 = w.y / p->Nr;
    return;
  }
  const TcPass& P = T->pass[w.x];
  const int half = p->Nph / 2;
  auto field = [&](long long vg) {
    if (w.x == tcx::kItemTheta) return P.h_list[(size_t)(vg / half)] / p->Nr;
    return P.h_list[(size_t)vg] / p->Nth / p->Nr;
  };
  *f0 = field(w.y);
  *f1 = field((long long)w.y + w.z - 1);
}
}  // namespace

cudaError_t tc_launch(sph_filter_plan_s* p, const double* in, double* out, int transpose, int var_begin,
                      int var_count, cudaStream_t s, int, int* nlaunch) {
  int dummy = 0;
  if (!nlaunch) nlaunch = &dummy;
  *nlaunch = 0;
  TcPlan* T = p->tc;
  const int4* items = T->d_items;
  int n_fused = T->n_fused, n_theta = T->n_theta, n_phi = T->n_phi;
  if (var_begin != 0 || var_count != p->nvars) {
    // a field range (e.g. one chunk of the host-buffer pipeline): the items that touch it
    std::lock_guard<std::mutex> lock(T->mu);
    auto it = T->ranges.find({var_begin, var_count});
    if (it == T->ranges.end()) {
      TcPlan::RangeItems R;
      std::vector<int4> sel;
      const int ve = var_begin + var_count;
      const int bounds[4] = {0, T->n_fused, T->n_fused + T->n_theta, T->n_fused + T->n_theta + T->n_phi};
      int counts[3] = {0, 0, 0};
      for (int part = 0; part < 3; ++part)
        for (int i = bounds[part]; i < bounds[part + 1]; ++i) {
          int f0, f1;
          item_fields(p, T->h_items[(size_t)i], &f0, &f1);
          if (f1 < var_begin || f0 >= ve) continue;
          sel.push_back(T->h_items[(size_t)i]);
          ++counts[part];
        }
      if (!sel.empty()) {
        if (cudaMalloc((void**)&R.d, sel.size() * sizeof(int4)) != cudaSuccess) return cudaErrorMemoryAllocation;
        const cudaError_t e = cudaMemcpy(R.d, sel.data(), sel.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
      }
      R.n_fused = counts[0];
      R.n_theta = counts[1];
      R.n_phi = counts[2];
      it = T->ranges.emplace(std::make_pair(var_begin, var_count), R).first;
    }
    items = it->second.d;
    n_fused = it->second.n_fused;
    n_theta = it->second.n_theta;
    n_phi = it->second.n_phi;
  }
  if (!transpose) {
    // one launch: theta tiles in -> out, phi tiles of shells with a theta pass out -> out after them,
    // the others in -> out, and copies of the rings no pass changes (Sec. II.C order)
    return launch_items(p, items, n_fused, 1, in, out, var_begin, var_count, s, nlaunch);
  }
  // transpose: phi pass, then theta pass, both in place on out
  const size_t field = (size_t)p->Nth * p->Nph * p->Nr;
  if (in != out) {
    const cudaError_t e = cudaMemcpyAsync(out + field * var_begin, in + field * var_begin,
                                          sizeof(double) * field * var_count, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = launch_items(p, items + n_fused + n_theta, n_phi, 0, out, out, var_begin, var_count, s, nlaunch);
  if (e != cudaSuccess) return e;
  return launch_items(p, items + n_fused, n_theta, 0, out, out, var_begin, var_count, s, nlaunch);
}

// ---------------------------------------------------------------- several plans in one launch

struct TcBatch {
  std::vector<sph_filter_plan_s*> plans;
  int4* d_items = nullptr;
  int nitems = 0;
  int* d_counters = nullptr;        // [0, 2) work, then each grid's circles
  std::vector<size_t> circ_off;
  tcx::KShape shape{};
  int threads = 0, ctas_per_sm = 1;
  size_t smem = 0;
};

sph_status tc_batch_setup(TcBatch** out, sph_filter_plan_s* const* plans, int nplans) {
  *out = nullptr;
  if (nplans < 1 || nplans > tcx::kMaxGrids) return SPH_EUNSUPPORTED;
  TcBatch* B = new (std::nothrow) TcBatch();
  if (!B) return SPH_ENOMEM;
  // items of every grid, each phase of the fused order merged over the grids, costliest tiles first
  struct It {
    int4 w;
    long long cost;
  };
  std::vector<It> ph[3];
  size_t circ = 2;
  int ctas = 2;
  for (int g = 0; g < nplans; ++g) {
    sph_filter_plan_s* p = plans[g];
    TcPlan* T = p->tc;
    B->plans.push_back(p);
    B->circ_off.push_back(circ);
    circ += (size_t)T->nshells;
    // the fused list: theta tiles, then phi tiles and copies without theta results, then the rest
    for (int i = 0; i < T->n_fused; ++i) {
      int4 w = T->h_items[(size_t)i];
      const int phase = w.x == tcx::kItemTheta ? 0 : (w.x == tcx::kItemPhi && w.w) ? 2 : 1;
      const long long cost = w.x == tcx::kItemCopy ? (long long)w.w * p->Nph / 8
                                                   : (long long)w.z * (w.x == tcx::kItemTheta ? 2 * p->Nth : p->Nph);
      w.x |= g << 4;
      ph[phase].push_back(It{w, cost});
    }
    B->shape.Lmax = std::max(B->shape.Lmax, T->shape.Lmax);
    B->shape.opmax = std::max(B->shape.opmax, T->shape.opmax);
    B->shape.tmem_cols = std::max(B->shape.tmem_cols, T->shape.tmem_cols);
    B->threads = std::max(B->threads, T->threads);
    ctas = std::min(ctas, T->ctas_per_sm);
  }
  std::vector<int4> items;
  for (auto& v : ph) {
    std::stable_sort(v.begin(), v.end(), [](const It& a, const It& b) { return a.cost > b.cost; });
    for (const It& x : v) items.push_back(x.w);
  }
  B->nitems = (int)items.size();
  const int device = plans[0]->device;
  const int optin = max_smem_optin(device);
  B->smem = ((size_t)B->shape.opmax + 1023) / 1024 * 1024 + (size_t)tcx::kV * (B->shape.Lmax + 1) * 8 + sizeof(tcx::Ctl);
  if ((int)B->smem > optin) {
    delete B;
    return SPH_EUNSUPPORTED;
  }
  B->ctas_per_sm = (ctas == 2 && B->shape.tmem_cols <= 256 && B->threads <= 256 && 2 * (B->smem + 1024) <= (size_t)optin) ? 2 : 1;
  B->smem = std::min(std::max(B->smem, (size_t)optin / (B->ctas_per_sm + 1) + 1024), (size_t)optin);
  bool ok = cudaMalloc((void**)&B->d_items, items.size() * sizeof(int4)) == cudaSuccess &&
            cudaMemcpy(B->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMalloc((void**)&B->d_counters, circ * sizeof(int)) == cudaSuccess &&
            cudaMemset(B->d_counters, 0, circ * sizeof(int)) == cudaSuccess &&
            cudaFuncSetAttribute(tcx::tc_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem) ==
                cudaSuccess;
  if (!ok) {
    tc_batch_free(B);
    return SPH_ECUDA;
  }
  *out = B;
  return SPH_OK;
}

void tc_batch_free(TcBatch* B) {
  if (!B) return;
  cudaFree(B->d_items);
  cudaFree(B->d_counters);
  delete B;
}

cudaError_t tc_batch_launch(TcBatch* B, const double* const* in, double* const* out, cudaStream_t s) {
  tcx::BatchArgs ba{};
  ba.ngrids = (int)B->plans.size();
  for (int g = 0; g < ba.ngrids; ++g) {
    sph_filter_plan_s* p = B->plans[(size_t)g];
    ba.g[g] = plan_args(p, 1, in[g], out[g], 0, p->nvars);
    ba.g[g].circles = B->d_counters + B->circ_off[(size_t)g];
  }
  ba.shape = B->shape;
  ba.items = B->d_items;
  ba.nitems = B->nitems;
  ba.work = B->d_counters;
  const int nsm = B->plans[0]->tc->nsm;
  const int grid = std::min(B->nitems, nsm * B->ctas_per_sm);
  if (grid <= 0) return cudaSuccess;
  tcx::tc_batch_kernel<<<grid, B->threads, B->smem, s>>>(ba);
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) B->plans[0]->launched += 1;
  return e;
}

}  // namespace sph
