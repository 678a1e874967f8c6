// Algebraic-constraint map applied after filtering (Sec. II.C, "Filtering spacetime fields in the
// presence of BHs"): at every point the conformal metric is rescaled so that its determinant equals
// the background's, and the trace of the conformal extrinsic curvature is removed; where the theta
// filter is active and the lapse is below a threshold (0.3 in the paper), only h_11 is solved from
// the determinant condition and A is kept.
//
// Components are orthonormal-basis components, h_{ab} (gamma_bar_ij = R_i R_j (delta_ij + h_ij) for
// the spherical scale factors R = (1, r, r sin theta)) and A_{ab}. The scale factors cancel from
// both constraints, so the map acts on m = delta + h and A alone, point by point.
//
// One thread per point, grid-stride over a grid of 8 CTAs per SM: every field plane is read with
// unit stride. The standard form runs in compensated FP32 pairs (about 48-bit significands: FP32
// instructions instead of the slow FP64 pipe); the modified form, and points with a value outside
// the pairs' range, run in FP64.
#include <cmath>
#include <cstdint>

#include "df32.h"
#include "internal.h"

namespace {

struct ConstraintVars {
  int h[6];  // field index of h_11, h_12, h_13, h_22, h_23, h_33
  int a[6];  // field index of A_11, ..., A_33 (same order)
  int alpha;
};

using sph::df;

// Compensated FP32-pair arithmetic (error-free transformations: Knuth's TwoSum, the FMA product).
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return df{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df dadd(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return renorm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df dneg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ df dmul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return renorm(p, e);
}
__device__ __forceinline__ df dmulf(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return renorm(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
// a / b: three quotient terms from the rounded FP32 reciprocal of b.hi, each remainder formed exactly.
__device__ __forceinline__ df ddiv(df a, df b) {
  const float y = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, y);
  const df r1 = dsub(a, dmulf(b, q1));
  const float q2 = __fmul_rn(r1.hi, y);
  const df r2 = dsub(r1, dmulf(b, q2));
  const float q3 = __fmul_rn(r2.hi, y);
  const df q = two_sum(q1, q2);
  return renorm(q.hi, __fadd_rn(q.lo, q3));
}

// A value's biased FP64 exponent field in the range where the pair conversions keep full relative
// precision (the low part a normal FP32 number) and the products and the cube root stay far from
// FP32 overflow; zero passes too.
__device__ __forceinline__ bool pair_range(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return e == 0 || (e >= 1023 - 70 && e <= 1023 + 40);
}

__global__ void __launch_bounds__(256) constraint_kernel(double* __restrict__ s, ConstraintVars v,
                                                          const unsigned char* __restrict__ theta_filtered,
                                                          long long plane, long long shell_points,
                                                          double alpha_bh) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += stride) {
    double* hp[6];
    double h[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) {
      hp[n] = s + (size_t)v.h[n] * (size_t)plane + p;
      h[n] = *hp[n];
    }
    const double alpha = s[(size_t)v.alpha * (size_t)plane + p];
    if (theta_filtered && theta_filtered[p / shell_points] && alpha < alpha_bh) {
      // modified form (FP64): det(m) = 1 solved for m_11 with the other components kept; A unchanged
      const double m12 = h[1], m13 = h[2], m22 = 1.0 + h[3], m23 = h[4], m33 = 1.0 + h[5];
      const double c11 = m22 * m33 - m23 * m23;
      *hp[0] = (1.0 + m12 * m12 * m33 - 2.0 * m12 * m13 * m23 + m13 * m13 * m22) / c11 - 1.0;
      continue;
    }
    double* ap[6];
    double a[6];
    bool pr = true;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
      ap[n] = s + (size_t)v.a[n] * (size_t)plane + p;
      a[n] = *ap[n];
      pr = pr && pair_range(h[n]) && pair_range(a[n]);
    }
    if (pr) {
      // standard form in compensated FP32 pairs (m = delta + h, its cofactors, det, the trace of A
      // in m, det^(-1/3) by two Newton steps from the FP32 estimate, kept as det^(-1/3) - 1 so that
      // h' = (sc - 1) + sc h keeps its relative accuracy for small h)
      df hd[6], ad[6];
#pragma unroll
      for (int n = 0; n < 6; ++n) {
        hd[n] = sph::df_from_double(h[n], 0);
        ad[n] = sph::df_from_double(a[n], 0);
      }
      const df one{1.0f, 0.0f};
      const df m11 = dadd(one, hd[0]), m12 = hd[1], m13 = hd[2];
      const df m22 = dadd(one, hd[3]), m23 = hd[4], m33 = dadd(one, hd[5]);
      const df c11 = dsub(dmul(m22, m33), dmul(m23, m23));
      const df c12 = dsub(dmul(m13, m23), dmul(m12, m33));
      const df c13 = dsub(dmul(m12, m23), dmul(m13, m22));
      const df c22 = dsub(dmul(m11, m33), dmul(m13, m13));
      const df c23 = dsub(dmul(m12, m13), dmul(m11, m23));
      const df c33 = dsub(dmul(m11, m22), dmul(m12, m12));
      const df det = dadd(dadd(dmul(m11, c11), dmul(m12, c12)), dmul(m13, c13));
      df num = dadd(dadd(dmul(c11, ad[0]), dmul(c22, ad[3])), dmul(c33, ad[5]));
      const df off = dadd(dadd(dmul(c12, ad[1]), dmul(c13, ad[2])), dmul(c23, ad[4]));
      num = dadd(num, dadd(off, off));
      const df t3 = dmul(ddiv(num, det), df{0.333333343f, -9.93410776e-09f});  // 1/3 as a pair
      const float y0 = rcbrtf(det.hi);
      // y <- y + y (1 - det y^3) / 3, twice; d = y - y0 accumulated as a pair
      df d{0.0f, 0.0f};
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const df y = dadd(df{y0, 0.0f}, d);
        const df e = dsub(one, dmul(det, dmul(y, dmul(y, y))));
        d = dadd(d, dmul(y, dmul(e, df{0.333333343f, -9.93410776e-09f})));
      }
      const df sc = dadd(df{y0, 0.0f}, d);
      const df scm1 = dadd(two_sum(y0, -1.0f), d);  // y0 - 1 is exact
      const df mab[6] = {m11, m12, m13, m22, m23, m33};
#pragma unroll
      for (int n = 0; n < 6; ++n) {
        const bool diag = n == 0 || n == 3 || n == 5;
        const df hs = dmul(sc, hd[n]);
        *hp[n] = sph::df_to_double(diag ? dadd(scm1, hs) : hs, 0);
        *ap[n] = sph::df_to_double(dsub(ad[n], dmul(mab[n], t3)), 0);
      }
      continue;
    }
    // standard form in FP64 (values outside the pair range)
    const double m11 = 1.0 + h[0], m12 = h[1], m13 = h[2];
    const double m22 = 1.0 + h[3], m23 = h[4], m33 = 1.0 + h[5];
    // cofactors of the symmetric m (c_ab = c_ba)
    const double c11 = m22 * m33 - m23 * m23, c12 = m13 * m23 - m12 * m33, c13 = m12 * m23 - m13 * m22;
    const double c22 = m11 * m33 - m13 * m13, c23 = m12 * m13 - m11 * m23, c33 = m11 * m22 - m12 * m12;
    const double det = m11 * c11 + m12 * c12 + m13 * c13;
    // trace of A in the metric m: sum (m^-1)_ab A_ab, m^-1 = cofactors / det. A loses m tr / 3,
    // which equals m' tr' / 3 for the rescaled metric m' = det^(-1/3) m.
    const double tr = (c11 * a[0] + c22 * a[3] + c33 * a[5] + 2.0 * (c12 * a[1] + c13 * a[2] + c23 * a[4])) / det;
    const double t3 = tr / 3.0;
    const double sc = rcbrt(det);
    *hp[0] = sc * m11 - 1.0;
    *hp[1] = sc * m12;
    *hp[2] = sc * m13;
    *hp[3] = sc * m22 - 1.0;
    *hp[4] = sc * m23;
    *hp[5] = sc * m33 - 1.0;
    *ap[0] = a[0] - m11 * t3;
    *ap[1] = a[1] - m12 * t3;
    *ap[2] = a[2] - m13 * t3;
    *ap[3] = a[3] - m22 * t3;
    *ap[4] = a[4] - m23 * t3;
    *ap[5] = a[5] - m33 * t3;
  }
}

}  // namespace

extern "C" sph_status sph_enforce_constraints(double* state, int nvars, int Nr, int Ntheta, int Nphi,
                                              const int* h_vars, const int* a_vars, int alpha_var,
                                              const unsigned char* theta_filtered, double alpha_bh,
                                              sph_stream_t stream) {
  if (!state || !h_vars || !a_vars || nvars < 13 || Nr < 1 || Ntheta < 1 || Nphi < 1 || !std::isfinite(alpha_bh))
    return SPH_EINVAL;
  if ((uintptr_t)state % alignof(double) != 0) return SPH_EINVAL;
  ConstraintVars v{};
  int idx[13];
  for (int n = 0; n < 6; ++n) {
    idx[n] = v.h[n] = h_vars[n];
    idx[6 + n] = v.a[n] = a_vars[n];
  }
  idx[12] = v.alpha = alpha_var;
  for (int n = 0; n < 13; ++n) {
    if (idx[n] < 0 || idx[n] >= nvars) return SPH_EINVAL;
    for (int k = 0; k < n; ++k)
      if (idx[k] == idx[n]) return SPH_EINVAL;  // the 13 fields must be distinct
  }
  const long long shell_points = (long long)Ntheta * Nphi, plane = (long long)Nr * shell_points;
  // both arrays must live on the current device: the kernel runs there and would otherwise touch
  // another GPU's memory
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPH_ECUDA;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, state) != cudaSuccess) return SPH_ECUDA;
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return SPH_EINVAL;
  if (attr.type == cudaMemoryTypeDevice && attr.device != dev) return SPH_EINVAL;
  if (theta_filtered) {
    if (cudaPointerGetAttributes(&attr, theta_filtered) != cudaSuccess) return SPH_ECUDA;
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return SPH_EINVAL;
    if (attr.type == cudaMemoryTypeDevice && attr.device != dev) return SPH_EINVAL;
  }
  const long long want = (plane + 255) / 256, cap = 8LL * sms;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  constraint_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(state, v, theta_filtered, plane, shell_points, alpha_bh);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
}
