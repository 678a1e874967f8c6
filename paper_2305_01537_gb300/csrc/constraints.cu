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
// unit stride. The arithmetic is FP64 (about 70 flops and one reciprocal cube root per point).
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace {

struct ConstraintVars {
  int h[6];  // field index of h_11, h_12, h_13, h_22, h_23, h_33
  int a[6];  // field index of A_11, ..., A_33 (same order)
  int alpha;
};

__global__ void __launch_bounds__(256) constraint_kernel(double* __restrict__ s, ConstraintVars v,
                                                          const unsigned char* __restrict__ theta_filtered,
                                                          long long plane, long long shell_points,
                                                          double alpha_bh) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += stride) {
    double* hp[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) hp[n] = s + (size_t)v.h[n] * (size_t)plane + p;
    const double m11 = 1.0 + *hp[0], m12 = *hp[1], m13 = *hp[2];
    const double m22 = 1.0 + *hp[3], m23 = *hp[4], m33 = 1.0 + *hp[5];
    const double alpha = s[(size_t)v.alpha * (size_t)plane + p];
    // cofactors of the symmetric m (c_ab = c_ba)
    const double c11 = m22 * m33 - m23 * m23, c12 = m13 * m23 - m12 * m33, c13 = m12 * m23 - m13 * m22;
    if (theta_filtered && theta_filtered[p / shell_points] && alpha < alpha_bh) {
      // modified form: det(m) = 1 solved for m_11 with the other components kept; A unchanged
      *hp[0] = (1.0 + m12 * m12 * m33 - 2.0 * m12 * m13 * m23 + m13 * m13 * m22) / c11 - 1.0;
      continue;
    }
    const double c22 = m11 * m33 - m13 * m13, c23 = m12 * m13 - m11 * m23, c33 = m11 * m22 - m12 * m12;
    const double det = m11 * c11 + m12 * c12 + m13 * c13;
    double* ap[6];
    double a[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) {
      ap[n] = s + (size_t)v.a[n] * (size_t)plane + p;
      a[n] = *ap[n];
    }
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
