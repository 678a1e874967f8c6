// Plain form of the double FFT filter (arXiv:2305.01537, Sec. II.C): FP64 arithmetic, one CTA per
// (field, shell). The whole Ntheta x Nphi shell is staged in shared memory, so both passes cost one
// HBM read and one HBM write of the shell.
//
// theta pass (Sec. II.C, first filter equation and the double covering): for each meridian pair
//   (k, k + Nphi/2) the circle c[q] = x[q][k] (q < Ntheta), (-1)^a x[2 Ntheta - 1 - q][k + Nphi/2]
//   (q >= Ntheta) is transformed, multiplied by f(|l|, l_max) and transformed back. Two real
//   circles share one complex FFT (real part / imaginary part): their multipliers are equal, and a
//   real even multiplier maps real sequences to real sequences.
// phi pass (Sec. II.C, second filter equation): every active ring is transformed, multiplied by
//   f(|m|, m_max(r, theta_j)) and transformed back. Two rings share one complex FFT Z = X1 + i X2;
//   with their (different) real even multipliers f1, f2 the filtered pair is the inverse FFT of
//   W_m = (f1+f2)/2 Z_m + (f1-f2)/2 conj(Z_{-m}).
// Identity skipping: with the exponential or the sharp filter a circle is unchanged when
//   l_max >= Ntheta (every |l| <= Ntheta is kept with factor 1) and a ring when m_max >= Nphi/2.
//   Those shells and rings are copied, which is exact.
//
// FFTs are mixed-radix Stockham transforms (radix 8, 4, 2, 3 hand-written, any other prime up to
// 64 by a direct DFT), batched over sequences, ping-ponging between two shared-memory buffers.
#include <cstdio>

#include "internal.h"

namespace sph {

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// multiply by DIR * i (DIR = -1 forward, +1 inverse)
template <int DIR>
__device__ __forceinline__ double2 mul_i(double2 v) {
  return DIR < 0 ? make_double2(v.y, -v.x) : make_double2(-v.y, v.x);
}

// In-register DFT of R points, V[u] = sum_r v[r] exp(DIR 2 pi i u r / R).
template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<2, DIR> {
  static __device__ __forceinline__ void run(double2* v) {
    double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR>
struct Dft<4, DIR> {
  static __device__ __forceinline__ void run(double2* v) {
    double2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    double2 c = cadd(v[1], v[3]), d = mul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <int DIR>
struct Dft<8, DIR> {
  static __device__ __forceinline__ void run(double2* v) {
    double2 e[4] = {v[0], v[2], v[4], v[6]};
    double2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, DIR>::run(e);
    Dft<4, DIR>::run(o);
    const double c = 0.70710678118654752440;  // sqrt(1/2)
    // o[u] *= w8^u, w8 = exp(DIR i pi / 4)
    double2 o1 = make_double2(c * (o[1].x - DIR * o[1].y), c * (o[1].y + DIR * o[1].x));
    double2 o2 = mul_i<DIR>(o[2]);
    double2 o3 = make_double2(c * (-o[3].x - DIR * o[3].y), c * (-o[3].y + DIR * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <int DIR>
struct Dft<3, DIR> {
  static __device__ __forceinline__ void run(double2* v) {
    const double h = 0.86602540378443864676;  // sqrt(3)/2
    double2 t = cadd(v[1], v[2]);
    double2 s = csub(v[1], v[2]);
    double2 m = make_double2(v[0].x - 0.5 * t.x, v[0].y - 0.5 * t.y);
    double2 w = mul_i<DIR>(make_double2(h * s.x, h * s.y));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, w);
    v[2] = csub(m, w);
  }
};

// One Stockham stage of radix R over a batch of B sequences of length N stored back to back.
// Ns is the product of the radices of the stages already done. tw[n] = exp(-2 pi i n / N).
template <int R, int DIR>
__device__ void stage(const double2* __restrict__ in, double2* __restrict__ out, int N, int B, int Ns,
                      const double2* __restrict__ tw) {
  const int NR = N / R;
  const int tws = N / (Ns * R);
  for (int w = threadIdx.x; w < B * NR; w += blockDim.x) {
    const int b = w / NR, j = w - b * NR;
    const int k = j % Ns;
    const double2* src = in + b * N + j;
    double2 v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = src[t * NR];
    if (Ns > 1) {
#pragma unroll
      for (int t = 1; t < R; ++t) {
        double2 wt = tw[t * k * tws];
        if (DIR > 0) wt.y = -wt.y;
        v[t] = cmul(v[t], wt);
      }
    }
    Dft<R, DIR>::run(v);
    double2* dst = out + b * N + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int t = 0; t < R; ++t) dst[t * Ns] = v[t];
  }
}

constexpr int kMaxGenericRadix = 64;

// Stage of any radix R <= 64 (a direct DFT of R points; used for primes other than 2 and 3).
template <int DIR>
__device__ void stage_generic(const double2* __restrict__ in, double2* __restrict__ out, int N, int B,
                              int Ns, int R, const double2* __restrict__ tw) {
  const int NR = N / R;
  const int tws = N / (Ns * R);
  for (int w = threadIdx.x; w < B * NR; w += blockDim.x) {
    const int b = w / NR, j = w - b * NR;
    const int k = j % Ns;
    const double2* src = in + b * N + j;
    double2 v[kMaxGenericRadix];
    for (int t = 0; t < R; ++t) {
      double2 x = src[t * NR];
      if (Ns > 1 && t > 0) {
        double2 wt = tw[t * k * tws];
        if (DIR > 0) wt.y = -wt.y;
        x = cmul(x, wt);
      }
      v[t] = x;
    }
    double2* dst = out + b * N + (j / Ns) * Ns * R + k;
    for (int u = 0; u < R; ++u) {
      double2 acc = make_double2(0.0, 0.0);
      for (int t = 0; t < R; ++t) {
        double2 wt = tw[((u * t) % R) * NR];
        if (DIR > 0) wt.y = -wt.y;
        acc = cadd(acc, cmul(v[t], wt));
      }
      dst[u * Ns] = acc;
    }
  }
}

// Batched FFT; returns the buffer that holds the result (a or b).
template <int DIR>
__device__ double2* fft(double2* a, double2* b, int N, int B, const Factors& f, const double2* tw) {
  double2* src = a;
  double2* dst = b;
  int Ns = 1;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.radix[s];
    switch (R) {
      case 8: stage<8, DIR>(src, dst, N, B, Ns, tw); break;
      case 4: stage<4, DIR>(src, dst, N, B, Ns, tw); break;
      case 2: stage<2, DIR>(src, dst, N, B, Ns, tw); break;
      case 3: stage<3, DIR>(src, dst, N, B, Ns, tw); break;
      default: stage_generic<DIR>(src, dst, N, B, Ns, R, tw); break;
    }
    __syncthreads();
    double2* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

// Filter function f(|l|, l_max) of Sec. II.C; `al` is |l|.
__device__ __forceinline__ double filter_value(int kind, double al, double lmax) {
  if (kind == SPH_FILTER_GAUSS) {
    const double t = al / (lmax + 1.0);
    return exp(-0.10536051565782630123 * t * t);  // log(0.9) = -0.1053605156578263...
  }
  if (al <= lmax) return 1.0;
  return kind == SPH_FILTER_EXP ? exp(-(al - lmax)) : 0.0;
}

struct Smem {
  double* S;        // staged shell, Nth rows of stride ldS
  double2* tw_th;   // 2 Nth
  double2* tw_ph;   // Nph
  double* g_th;     // Nth + 1 theta multipliers (already divided by 2 Nth)
  int* rings;       // active ring list, Nth entries (+1 count slot)
  double2* buf0;
  double2* buf1;
};

__device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__device__ Smem carve(const ShellArgs& A, unsigned char* base) {
  Smem m;
  size_t off = 0;
  m.S = reinterpret_cast<double*>(base + off);
  off = align_up(off + sizeof(double) * (size_t)A.Nth * A.ldS, 16);
  m.tw_th = reinterpret_cast<double2*>(base + off);
  off += sizeof(double2) * 2 * A.Nth;
  m.tw_ph = reinterpret_cast<double2*>(base + off);
  off += sizeof(double2) * A.Nph;
  m.g_th = reinterpret_cast<double*>(base + off);
  off = align_up(off + sizeof(double) * (A.Nth + 1), 16);
  m.rings = reinterpret_cast<int*>(base + off);
  off = align_up(off + sizeof(int) * (A.Nth + 1), 16);
  const size_t nb = (size_t)max(A.chunk_th * 2 * A.Nth, A.chunk_ph * A.Nph);
  m.buf0 = reinterpret_cast<double2*>(base + off);
  m.buf1 = m.buf0 + nb;
  return m;
}

__device__ void theta_pass(const ShellArgs& A, const Smem& m, int parity, int kind, double lmax) {
  if (kind != SPH_FILTER_GAUSS && lmax >= (double)A.Nth) return;  // every |l| <= Ntheta kept
  const int Nth = A.Nth, M = 2 * Nth, half = A.Nph / 2, ld = A.ldS;
  const double sgn = parity ? -1.0 : 1.0;
  const double invM = 1.0 / (double)M;
  for (int l = threadIdx.x; l <= Nth; l += blockDim.x) m.g_th[l] = filter_value(kind, (double)l, lmax) * invM;
  const int nseq = (half + 1) / 2;  // circles k = 2s and 2s+1 share sequence s
  for (int s0 = 0; s0 < nseq; s0 += A.chunk_th) {
    const int B = min(A.chunk_th, nseq - s0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < B * M; idx += blockDim.x) {
      const int b = idx / M, q = idx - b * M;
      const int k1 = 2 * (s0 + b), k2 = k1 + 1;
      double re, im = 0.0;
      if (q < Nth) {
        re = m.S[q * ld + k1];
        if (k2 < half) im = m.S[q * ld + k2];
      } else {
        const int j = M - 1 - q;
        re = sgn * m.S[j * ld + k1 + half];
        if (k2 < half) im = sgn * m.S[j * ld + k2 + half];
      }
      m.buf0[idx] = make_double2(re, im);
    }
    __syncthreads();
    double2* X = fft<-1>(m.buf0, m.buf1, M, B, A.f_th, m.tw_th);
    for (int idx = threadIdx.x; idx < B * M; idx += blockDim.x) {
      const int l = idx % M;
      const double g = m.g_th[l <= Nth ? l : M - l];
      X[idx] = make_double2(X[idx].x * g, X[idx].y * g);
    }
    __syncthreads();
    double2* Y = fft<1>(X, X == m.buf0 ? m.buf1 : m.buf0, M, B, A.f_th, m.tw_th);
    for (int idx = threadIdx.x; idx < B * Nth; idx += blockDim.x) {
      const int b = idx / Nth, j = idx - b * Nth;
      const int k1 = 2 * (s0 + b), k2 = k1 + 1;
      const double2 lo = Y[b * M + j];
      const double2 hi = Y[b * M + M - 1 - j];
      m.S[j * ld + k1] = lo.x;
      m.S[j * ld + k1 + half] = sgn * hi.x;
      if (k2 < half) {
        m.S[j * ld + k2] = lo.y;
        m.S[j * ld + k2 + half] = sgn * hi.y;
      }
    }
  }
  __syncthreads();
}

__device__ void phi_pass(const ShellArgs& A, const Smem& m, int kind, const double* mmax_row) {
  const int Nth = A.Nth, N = A.Nph, ld = A.ldS;
  const double nyq = 0.5 * (double)N;
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int j = 0; j < Nth; ++j)
      if (kind == SPH_FILTER_GAUSS || mmax_row[j] < nyq) m.rings[n++] = j;
    m.rings[Nth] = n;
  }
  __syncthreads();
  const int nact = m.rings[Nth];
  const int npair = (nact + 1) / 2;
  const double invN = 1.0 / (double)N;
  for (int p0 = 0; p0 < npair; p0 += A.chunk_ph) {
    const int B = min(A.chunk_ph, npair - p0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < B * N; idx += blockDim.x) {
      const int b = idx / N, k = idx - b * N;
      const int a1 = 2 * (p0 + b), a2 = a1 + 1;
      const double re = m.S[m.rings[a1] * ld + k];
      const double im = (a2 < nact) ? m.S[m.rings[a2] * ld + k] : 0.0;
      m.buf0[idx] = make_double2(re, im);
    }
    __syncthreads();
    double2* X = fft<-1>(m.buf0, m.buf1, N, B, A.f_ph, m.tw_ph);
    const int nh = N / 2 + 1;
    for (int idx = threadIdx.x; idx < B * nh; idx += blockDim.x) {
      const int b = idx / nh, mm = idx - b * nh;
      const int a1 = 2 * (p0 + b), a2 = a1 + 1;
      const double mx1 = mmax_row[m.rings[a1]];
      const double mx2 = (a2 < nact) ? mmax_row[m.rings[a2]] : mx1;
      const double f1 = filter_value(kind, (double)mm, mx1);
      const double f2 = filter_value(kind, (double)mm, mx2);
      const double ca = 0.5 * (f1 + f2) * invN, cd = 0.5 * (f1 - f2) * invN;
      double2* Zb = X + b * N;
      const int mn = (N - mm) % N;
      const double2 zm = Zb[mm], zn = Zb[mn];
      const double2 wm = make_double2(ca * zm.x + cd * zn.x, ca * zm.y - cd * zn.y);
      if (mn == mm) {
        Zb[mm] = wm;
      } else {
        const double2 wn = make_double2(ca * zn.x + cd * zm.x, ca * zn.y - cd * zm.y);
        Zb[mm] = wm;
        Zb[mn] = wn;
      }
    }
    __syncthreads();
    double2* Y = fft<1>(X, X == m.buf0 ? m.buf1 : m.buf0, N, B, A.f_ph, m.tw_ph);
    for (int idx = threadIdx.x; idx < B * N; idx += blockDim.x) {
      const int b = idx / N, k = idx - b * N;
      const int a1 = 2 * (p0 + b), a2 = a1 + 1;
      const double2 y = Y[idx];
      m.S[m.rings[a1] * ld + k] = y.x;
      if (a2 < nact) m.S[m.rings[a2] * ld + k] = y.y;
    }
  }
  __syncthreads();
}

template <typename IO>
__global__ void __launch_bounds__(kThreads, 1) plain_shell_kernel(ShellArgs A, LaunchIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem m = carve(A, smem_raw);
  const int shell = io.var_begin * A.Nr + blockIdx.x;
  const int v = shell / A.Nr, i = shell - v * A.Nr;
  const VarInfo vi = A.var[v];
  const int Nth = A.Nth, Nph = A.Nph, ld = A.ldS;
  const size_t npts = (size_t)Nth * Nph;

  for (int n = threadIdx.x; n < 2 * Nth; n += blockDim.x) m.tw_th[n] = A.tw_th[n];
  for (int n = threadIdx.x; n < Nph; n += blockDim.x) m.tw_ph[n] = A.tw_ph[n];
  const IO* src = static_cast<const IO*>(io.in) + (size_t)shell * npts;
  for (int n = threadIdx.x; n < (int)npts; n += blockDim.x) {
    const int j = n / Nph, k = n - j * Nph;
    double x = (double)src[n];
    if (io.map_in == kMapTanh) x = tanh(x);
    m.S[j * ld + k] = x;
  }
  __syncthreads();

  const double lmax = A.lmax[vi.cls * A.Nr + i];
  const double* mmax_row = A.mmax + ((size_t)vi.cls * A.Nr + i) * Nth;
  if (!io.transpose) {
    theta_pass(A, m, vi.parity, vi.kind, lmax);
    phi_pass(A, m, vi.kind, mmax_row);
  } else {
    phi_pass(A, m, vi.kind, mmax_row);
    theta_pass(A, m, vi.parity, vi.kind, lmax);
  }
  __syncthreads();

  IO* dst = static_cast<IO*>(io.out) + (size_t)shell * npts;
  const IO* aux = io.map_out == kOutTanhGrad ? static_cast<const IO*>(io.aux) + (size_t)shell * npts : nullptr;
  for (int n = threadIdx.x; n < (int)npts; n += blockDim.x) {
    const int j = n / Nph, k = n - j * Nph;
    double y = m.S[j * ld + k];
    if (io.map_out == kOutTanhGrad) {
      const double t = tanh((double)aux[n]);
      y *= (1.0 - t * t);
    }
    dst[n] = (IO)y;
  }
}

}  // namespace

size_t plain_smem_bytes(const ShellArgs& a, int* chunk_th, int* chunk_ph) {
  auto up = [](size_t x, size_t al) { return (x + al - 1) / al * al; };
  size_t fixed = up(sizeof(double) * (size_t)a.Nth * a.ldS, 16);
  fixed += sizeof(double2) * (2 * (size_t)a.Nth + a.Nph);
  fixed = up(fixed + sizeof(double) * (a.Nth + 1), 16);
  fixed = up(fixed + sizeof(int) * (a.Nth + 1), 16);
  const int nseq_th = (a.Nph / 2 + 1) / 2;
  const int npair_ph = (a.Nth + 1) / 2;
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t budget = (size_t)max_smem_optin(dev);
  if (fixed >= budget) return 0;
  const size_t room = (budget - fixed) / (2 * sizeof(double2));  // complex slots per buffer
  int cth = (int)std::min<size_t>((size_t)nseq_th, room / (2 * (size_t)a.Nth));
  int cph = (int)std::min<size_t>((size_t)npair_ph, room / (size_t)a.Nph);
  if (cth < 1 || cph < 1) return 0;
  *chunk_th = cth;
  *chunk_ph = cph;
  const size_t nb = std::max((size_t)cth * 2 * a.Nth, (size_t)cph * a.Nph);
  return fixed + 2 * sizeof(double2) * nb;
}

cudaError_t launch_plain(const sph_filter_plan_s& p, const LaunchIO& io, cudaStream_t s) {
  const dim3 grid((unsigned)(io.var_count * p.Nr));
  if (io.is_f32) {
    plain_shell_kernel<float><<<grid, kThreads, p.smem_bytes, s>>>(p.args, io);
  } else {
    plain_shell_kernel<double><<<grid, kThreads, p.smem_bytes, s>>>(p.args, io);
  }
  return cudaGetLastError();
}

// The attribute is per kernel, not per plan: always raise it to the device's opt-in maximum so that
// no plan can lower it below what another plan launches with.
cudaError_t set_plain_smem_attr(size_t) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t bytes = (size_t)max_smem_optin(dev);
  e = cudaFuncSetAttribute(plain_shell_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(plain_shell_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sph
