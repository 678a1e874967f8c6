// C ABI of the double FFT filter library: plan creation (argument validation, FP64 cutoff and
// twiddle tables built on the host), the apply entry points and status handling.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "internal.h"

namespace sph {

int max_smem_per_sm(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess) return 0;
  return v;
}

int max_smem_optin(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
  return v;
}

cudaError_t set_plain_smem_attr(size_t bytes);


namespace {

// Radix order for a length: 8s, then 4, 2, 3, then any remaining prime (direct DFT stage).
bool factorize(int n, Factors* f) {
  f->n = n;
  f->nst = 0;
  int m = n;
  auto push = [&](int r) {
    if (f->nst >= kMaxStages) return false;
    f->radix[f->nst++] = r;
    m /= r;
    return true;
  };
  while (m % 8 == 0) if (!push(8)) return false;
  while (m % 4 == 0) if (!push(4)) return false;
  while (m % 2 == 0) if (!push(2)) return false;
  while (m % 3 == 0) if (!push(3)) return false;
  for (int p = 5; m > 1; p += 2) {
    while (m % p == 0) {
      if (p > 64) return false;  // the direct-DFT stage is limited to radix 64
      if (!push(p)) return false;
    }
    if ((long)p * p > m && m > 1) {
      if (m > 64) return false;
      if (!push(m)) return false;
    }
  }
  return true;
}

// exp(-2 pi i n / N) for n < N, evaluated in long double and rounded once.
std::vector<double2> twiddles(int N) {
  std::vector<double2> t((size_t)N);
  const long double twopi = 2.0L * acosl(-1.0L);
  for (int n = 0; n < N; ++n) {
    const long double a = twopi * (long double)n / (long double)N;
    t[(size_t)n] = make_double2((double)cosl(a), (double)(-sinl(a)));
  }
  return t;
}

// Cutoffs of Sec. II.C evaluated with the same double operations, in the same order, as the
// plain definition: l_max = max(floor, 2 r / dr_min L); m_max = max(floor, 2 r / dr_min sin(theta) L).
double lmax_of(double r, double dr_min, double L, double floor_) {
  const double v = 2 * r / dr_min * L;
  return v > floor_ ? v : floor_;
}
double mmax_of(double r, double dr_min, double L, double floor_, int j, int Nth) {
  const double pi = std::acos(-1.0);
  const double theta = ((double)j + 0.5) * pi / (double)Nth;
  const double v = 2 * r / dr_min * std::sin(theta) * L;
  return v > floor_ ? v : floor_;
}


// Filter function f(|l|, l_max) of Sec. II.C in extended precision (tables are rounded once). A
// hybrid field's own class holds the exponential filter (its Gaussian tables are another class).
long double fval(int kind, long double al, long double lmax) {
  if (kind == SPH_FILTER_HYBRID) kind = SPH_FILTER_EXP;
  if (kind == SPH_FILTER_GAUSS) {
    const long double t = al / (lmax + 1.0L);
    return expl(logl(0.9L) * t * t);
  }
  if (al <= lmax) return 1.0L;
  return kind == SPH_FILTER_EXP ? expl(-(al - lmax)) : 0.0L;
}

// Radices the staged shell kernel implements: 8, 4, 2, 3.
bool factorize_v2(int n, Factors* f) {
  f->n = n;
  f->nst = 0;
  int m = n;
  while (m > 1) {
    int r = (m % 8 == 0) ? 8 : (m % 4 == 0) ? 4 : (m % 2 == 0) ? 2 : (m % 3 == 0) ? 3 : 0;
    if (r == 0 || f->nst >= kMaxStages) return false;
    f->radix[f->nst++] = r;
    m /= r;
  }
  return true;
}

// Real values written either as FP64 or as FP32 pairs (hi, lo).
struct TabWriter {
  bool pair;
  std::vector<unsigned char>& buf;
  void real(size_t at, long double v) const {
    if (pair) {
      const float hi = (float)v;
      const float lo = (float)(v - (long double)hi);
      std::memcpy(&buf[at], &hi, 4);
      std::memcpy(&buf[at + 4], &lo, 4);
    } else {
      const double d = (double)v;
      std::memcpy(&buf[at], &d, 8);
    }
  }
};

// Builds the tables of the staged shell kernel; SPH_EUNSUPPORTED if the shape does not fit it.
sph_status setup_v2(sph_filter_plan_s* p) {
  ShellArgs2& a = p->args2;
  a.Nr = p->Nr;
  a.Nth = p->Nth;
  a.Nph = p->Nph;
  a.nvars = p->nvars;
  a.ldS = p->Nph + 2;  // even: value pairs are 16-byte aligned
  if (!factorize_v2(2 * p->Nth, &a.f_th) || !factorize_v2(p->Nph, &a.f_ph)) return SPH_EUNSUPPORTED;
  const bool spectral = p->precision == SPH_PREC_SPECTRAL;
  if (spectral && !factorize_v2(p->Nth, &a.f_sp)) return SPH_EUNSUPPORTED;
  // Two CTAs of 256 threads per SM when the shell plus a scratch batch fits half the shared memory
  // (their copies and barriers then overlap each other's arithmetic); otherwise one CTA of 512.
  const int nseq = (p->Nph / 2 + 1) / 2, npair = (p->Nth + 1) / 2;
  const size_t optin = (size_t)max_smem_optin(p->device);
  const size_t half_sm = (size_t)(max_smem_per_sm(p->device) / 2) - 1024;  // per-CTA reserve
  int threads = 0;
  size_t smem = 0;
  for (int pass = 0; pass < 2 && !threads; ++pass) {
    const size_t limit = pass == 0 ? std::min(half_sm, optin) : optin;
    for (int div = 1; div <= 64; div *= 2) {
      a.batch_th = std::max(1, (nseq + div - 1) / div);
      a.batch_ph = std::max(1, (npair + div - 1) / div);
      smem = shell_smem_bytes(a, p->precision);
      if (smem <= limit) {
        threads = pass == 0 ? 256 : 512;
        break;
      }
      if (a.batch_th == 1 && a.batch_ph == 1) break;
    }
  }
  if (!threads && p->Nth % 4 == 0 && p->Nph % 8 == 0) {
    // a cluster pair per shell: each CTA holds half of the columns (theta) or half of the rings
    // (phi); the halves are exchanged through distributed shared memory. The FFT scratch reuses
    // buffer memory that is free during each pass (see the kernel), which sets the batch sizes.
    const size_t ldc = (size_t)p->Nph / 2 + 2;
    const int nseq_cl = (p->Nph / 4 + 1) / 2, npair_cl = p->Nth / 4;
    const int cap_th = (int)((8 * (size_t)(p->Nth / 2) * ldc) / (16 * 2 * (size_t)p->Nth));
    const int cap_ph = (int)((8 * (size_t)(p->Nth / 4) * ldc) / (16 * (size_t)p->Nph));
    a.batch_th = std::min(nseq_cl, cap_th);
    a.batch_ph = std::min(npair_cl, 2 * cap_ph);
    smem = shell_smem_cl_bytes(a, p->precision);
    if (a.batch_th >= 1 && cap_ph >= 1 && smem <= optin) {
      threads = 512;
      p->cluster = true;
    }
  }
  if (!threads) return SPH_EUNSUPPORTED;

  const bool pair = p->precision == SPH_PREC_F32X2;
  const int Nr = p->Nr, Nth = p->Nth, Nph = p->Nph, nh = Nph / 2 + 1, ncls = p->ncls;
  const size_t n_ring = (size_t)ncls * Nr * Nth, n_gth = (size_t)ncls * Nr * (Nth + 1);
  const size_t n_gph = n_ring * nh;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_ring = 0;
  const size_t o_gth = up(o_ring + n_ring);
  const size_t o_gph = up(o_gth + 8 * n_gth);
  const size_t o_tth = up(o_gph + 8 * n_gph);
  const size_t o_tph = up(o_tth + 16 * (size_t)(2 * Nth));
  const size_t o_con = up(o_tph + 16 * (size_t)Nph);
  const size_t total = up(o_con + 16);
  std::vector<unsigned char> buf(total, 0);
  TabWriter W{pair, buf};
  const long double pi = acosl(-1.0L);
  for (int c = 0; c < ncls; ++c)
    for (int i = 0; i < Nr; ++i) {
      const double lm = p->h_lmax[(size_t)c * Nr + i];
      for (int l = 0; l <= Nth; ++l)
        W.real(o_gth + 8 * (((size_t)c * Nr + i) * (Nth + 1) + l), fval(p->cls_kind[c], l, lm) / (2.0L * Nth));
      for (int j = 0; j < Nth; ++j) {
        const double mm = p->h_mmax[((size_t)c * Nr + i) * Nth + j];
        const bool active = p->cls_kind[c] == SPH_FILTER_GAUSS || mm < 0.5 * Nph;
        buf[o_ring + ((size_t)c * Nr + i) * Nth + j] = active ? 1 : 0;
        for (int m = 0; m < nh; ++m)
          W.real(o_gph + 8 * ((((size_t)c * Nr + i) * Nth + j) * nh + m), fval(p->cls_kind[c], m, mm) / (long double)Nph);
      }
      // mirror rings share one complex FFT; flag pairs whose multipliers differ beyond rounding
      for (int j = 0; j < Nth / 2; ++j) {
        const int jj = Nth - 1 - j;
        const double m1 = p->h_mmax[((size_t)c * Nr + i) * Nth + j], m2 = p->h_mmax[((size_t)c * Nr + i) * Nth + jj];
        bool differ = false;
        for (int m = 0; m < nh && !differ; ++m) {
          const long double d = fval(p->cls_kind[c], m, m1) - fval(p->cls_kind[c], m, m2);
          differ = fabsl(d) > 4e-16L;
        }
        if (differ) {
          buf[o_ring + ((size_t)c * Nr + i) * Nth + j] |= 2;
          buf[o_ring + ((size_t)c * Nr + i) * Nth + jj] |= 2;
        }
      }
    }
  // twiddles stage by stage, in the order of the kernels' radix sequence: the stage that follows
  // Ns points already combined, with radix R, holds exp(-2 pi i t kk / (Ns R)) at entry
  // kk (R - 1) + t - 1 (kk < Ns, 1 <= t < R); the tables add up to N - 1 entries
  // FP64 kernels (every precision but compensated FP32) run their radix-2, -4 and -8 stages as
  // radix-2 butterfly levels with FMA-form twiddles: per kk the slots hold w^4, w^2, w, w omega
  // (R = 8), w^2, w (R = 4) or w (R = 2), w = exp(-2 pi i kk / (Ns R)), omega = exp(-2 pi i / 8),
  // each as (m, r): m (1 + i r) with m = Re z, r = Im z / Re z when |Re z| >= |Im z|, else
  // i m (1 + i r) with m = Im z, r = -Re z / Im z, marked by the lowest significand bit of m.
  const bool fma_form = !W.pair;
  auto fma_twiddle = [&](size_t at, long double ang) {  // z = exp(-i ang)
    const long double zr = cosl(ang), zi = -sinl(ang);
    const bool cot = fabsl(zi) > fabsl(zr);
    double m = cot ? (double)zi : (double)zr;
    const double r = cot ? (double)(-zr / zi) : (double)(zi / zr);
    uint64_t bits;
    std::memcpy(&bits, &m, 8);
    bits = (bits & ~1ull) | (cot ? 1ull : 0ull);
    std::memcpy(&m, &bits, 8);
    W.real(at, m);
    W.real(at + 8, r);
  };
  auto stage_twiddles = [&](size_t o, const Factors& f) {
    size_t e = 0;
    int Ns = 1;
    for (int s = 0; s < f.nst; ++s) {
      const int R = f.radix[s];
      if (fma_form && (R == 2 || R == 4 || R == 8)) {
        for (int kk = 0; kk < Ns; ++kk, e += R - 1) {
          const long double a1 = 2.0L * pi * (long double)kk / (long double)(Ns * R);  // w = exp(-i a1)
          if (R == 8) {
            fma_twiddle(o + 16 * e, 4 * a1);
            fma_twiddle(o + 16 * (e + 1), 2 * a1);
            fma_twiddle(o + 16 * (e + 2), a1);
            fma_twiddle(o + 16 * (e + 3), a1 + pi / 4);
          } else if (R == 4) {
            fma_twiddle(o + 16 * e, 2 * a1);
            fma_twiddle(o + 16 * (e + 1), a1);
          } else {
            fma_twiddle(o + 16 * e, a1);
          }
        }
      } else {
        for (int kk = 0; kk < Ns; ++kk)
          for (int q = 1; q < R; ++q, ++e) {
            const long double ang = 2.0L * pi * (long double)(q * kk) / (long double)(Ns * R);
            W.real(o + 16 * e, cosl(ang));
            W.real(o + 16 * e + 8, -sinl(ang));
          }
      }
      Ns *= R;
    }
  };
  stage_twiddles(o_tph, kernel_radices(a, Nph, p->precision));
  if (!spectral) {
    stage_twiddles(o_tth, kernel_radices(a, 2 * Nth, p->precision));
  } else {
    // the spectral form's theta-table space (2 Ntheta entries): the stage twiddles of its
    // length-Ntheta transforms, then e^{i pi l / Ntheta}, l < Ntheta (the theta pass on doubled
    // circles never runs in these plans)
    stage_twiddles(o_tth, a.f_sp);
    for (int l = 0; l < Nth; ++l) {
      const long double ang = pi * (long double)l / (long double)Nth;
      W.real(o_tth + 16 * (size_t)(Nth + l), cosl(ang));
      W.real(o_tth + 16 * (size_t)(Nth + l) + 8, sinl(ang));
    }
  }
  W.real(o_con, sqrtl(0.5L));
  W.real(o_con + 8, sqrtl(3.0L) / 2.0L);
  if (cudaMalloc(&p->d_tabs, total) != cudaSuccess) return SPH_ENOMEM;
  if (cudaMemcpy(p->d_tabs, buf.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) return SPH_ECUDA;
  if (set_shell_smem_attr(p->device) != cudaSuccess) return SPH_ECUDA;
  unsigned char* base = static_cast<unsigned char*>(p->d_tabs);
  a.ring_info = base + o_ring;
  a.g_th = base + o_gth;
  a.g_ph = base + o_gph;
  a.tw_th = base + o_tth;
  a.tw_ph = base + o_tph;
  a.consts = base + o_con;
  a.lmax = p->d_lmax;
  a.var = p->d_var;
  a.status = p->d_status;
  p->threads2 = threads;
  p->smem2 = smem;
  p->use_v2 = true;
  if (!p->cluster) {
    // sparse shells: exponential or sharp filter with l_max >= Ntheta (the theta pass keeps every
    // mode); their active ring pairs become units
    std::vector<int> dense, sparse, units;
    p->dense_off.assign((size_t)p->nvars + 1, 0);
    p->sparse_off.assign((size_t)p->nvars + 1, 0);
    p->units_off.assign((size_t)p->nvars + 1, 0);
    for (int v = 0; v < p->nvars; ++v) {
      const int c = p->var_cls[(size_t)v], kind = p->kind[(size_t)v];
      for (int i = 0; i < Nr; ++i) {
        const bool sp = (kind == SPH_FILTER_EXP || kind == SPH_FILTER_SHARP) && !(p->h_lmax[(size_t)c * Nr + i] < (double)Nth);
        if (!sp) {
          dense.push_back(i * p->nvars + v);  // the shell kernel's grid index over all variables
          continue;
        }
        sparse.push_back(v * Nr + i);
        for (int j = 0; j < (Nth + 1) / 2; ++j) {
          const size_t rb = o_ring + ((size_t)c * Nr + i) * Nth;
          if ((buf[rb + j] | buf[rb + (Nth - 1 - j)]) & 1) units.push_back((v * Nr + i) * Nth + j);
        }
      }
      p->dense_off[(size_t)v + 1] = (int)dense.size();
      p->sparse_off[(size_t)v + 1] = (int)sparse.size();
      p->units_off[(size_t)v + 1] = (int)units.size();
    }
    p->smem_units = units_smem_bytes(a, p->precision);
    // (32-bit unit codes and multiplier offsets)
    const bool fits = (long long)p->nvars * Nr * Nth < (1ll << 31) &&
                      (long long)p->ncls * Nr * Nth * (p->Nph / 2 + 1) < (1ll << 32);
    if (!sparse.empty() && fits && p->smem_units <= (size_t)max_smem_optin(p->device)) {
      auto up_list = [](int** d, const std::vector<int>& h) {
        if (cudaMalloc((void**)d, sizeof(int) * std::max<size_t>(h.size(), 1)) != cudaSuccess) return SPH_ENOMEM;
        if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
          return SPH_ECUDA;
        return SPH_OK;
      };
      sph_status st = up_list(&p->d_dense, dense);
      if (st == SPH_OK) st = up_list(&p->d_sparse, sparse);
      if (st == SPH_OK) st = up_list(&p->d_units, units);
      int prio_low = 0, prio_high = 0;
      if (st == SPH_OK && (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess ||
                           cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaStreamCreateWithPriority(&p->side_copy, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
                           cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&p->ev_copy, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess))
        st = SPH_ECUDA;
      if (st != SPH_OK) return st;
      p->split = true;
    }
  }
  return SPH_OK;
}

bool overlaps_partially(const void* a, const void* b, size_t bytes) {
  if (a == b) return false;
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

template <typename T>
sph_status upload(T** dst, const T* src, size_t n) {
  if (cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) return SPH_ENOMEM;
  if (n && cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice) != cudaSuccess) return SPH_ECUDA;
  return SPH_OK;
}

void free_plan(sph_filter_plan_s* p) {
  if (!p) return;
  cudaFree(p->d_lmax);
  cudaFree(p->d_mmax);
  cudaFree(p->d_var);
  cudaFree(p->d_tw_th);
  cudaFree(p->d_tw_ph);
  cudaFree(p->d_status);
  cudaFree(p->d_tabs);
  cudaFree(p->d_dense);
  cudaFree(p->d_sparse);
  cudaFree(p->d_units);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->side_copy) cudaStreamDestroy(p->side_copy);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_copy) cudaEventDestroy(p->ev_copy);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  tc_free(p);
  cudaFree(p->d_stage_in);
  cudaFree(p->d_stage_out);
  for (cudaStream_t s : p->pipe)
    if (s) cudaStreamDestroy(s);
  for (cudaStream_t s : {p->pipe_in, p->pipe_out})
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : {p->pipe_start, p->pipe_end})
    if (e) cudaEventDestroy(e);
  for (const std::vector<cudaEvent_t>* v : {&p->chunk_in, &p->chunk_done})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  delete p;
}

// True if ptr is device memory of a GPU other than `device` (the kernels run on the plan's device and
// would otherwise read or write a peer's memory).
bool on_other_device(const void* ptr, int device) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice && attr.device != device;
}

sph_status check_io(const sph_filter_plan_s* p, const void* in, const void* out, size_t elem) {
  if (!p || !in || !out) return SPH_EINVAL;
  const size_t bytes = elem * (size_t)p->nvars * p->Nr * p->Nth * p->Nph;
  if (overlaps_partially(in, out, bytes)) return SPH_EALIAS;
  if (on_other_device(in, p->device) || on_other_device(out, p->device)) return SPH_EINVAL;
  return SPH_OK;
}

}  // namespace

long double filter_value(int kind, long double al, long double lmax) { return fval(kind, al, lmax); }

sph_status launch_plan(sph_filter_plan_s* p, const void* in, const void* aux, void* out, int map_in, int map_out,
                       int transpose, int is_f32, cudaStream_t stream) {
  if (!p) return SPH_EINVAL;
  return launch_plan_vars(p, in, aux, out, map_in, map_out, transpose, is_f32, 0, p->nvars, stream);
}

sph_status launch_plan_vars(sph_filter_plan_s* p, const void* in, const void* aux, void* out, int map_in,
                            int map_out, int transpose, int is_f32, int var_begin, int var_count,
                            cudaStream_t stream, int tc_set) {
  if (!p || var_begin < 0 || var_count < 1 || var_begin + var_count > p->nvars) return SPH_EINVAL;
  sph_status st = check_io(p, in, out, is_f32 ? sizeof(float) : sizeof(double));
  if (st != SPH_OK) return st;
  if (map_out == kOutTanhGrad) {
    if (!aux) return SPH_EINVAL;
    if (aux == out) return SPH_EALIAS;
    st = check_io(p, aux, out, is_f32 ? sizeof(float) : sizeof(double));
    if (st != SPH_OK) return st;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return SPH_ECUDA;
  if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) return SPH_ECUDA;
  if (p->tc) {
    // the tensor-core form implements the plain FP64 filter and its transpose only
    if (map_in != kMapNone || map_out != kOutNone || is_f32) {
      if (cur != p->device) cudaSetDevice(cur);
      return SPH_EUNSUPPORTED;
    }
    // the form keeps no state between launches, so calls on any streams may overlap
    int nl = 0;
    const cudaError_t e = tc_launch(p, static_cast<const double*>(in), static_cast<double*>(out), transpose, var_begin,
                                    var_count, (cudaStream_t)stream, tc_set, &nl);
    if (e == cudaSuccess) p->launched += nl;
    if (cur != p->device) cudaSetDevice(cur);
    return e == cudaSuccess ? SPH_OK : SPH_ECUDA;
  }
  int hybrid = 0;
  for (int v = var_begin; v < var_begin + var_count; ++v) hybrid |= p->kind[(size_t)v] == SPH_FILTER_HYBRID;
  if (hybrid && (transpose || map_in != kMapNone || map_out != kOutNone)) {
    // the hybrid switch is nonlinear: neither its transpose nor the fused chain steps are defined
    if (cur != p->device) cudaSetDevice(cur);
    return SPH_EUNSUPPORTED;
  }
  LaunchIO io{in,        aux,       out, map_in, map_out, transpose, is_f32, ((uintptr_t)in % 16) == 0 ? 1 : 0,
              var_begin, var_count, hybrid, nullptr, 0};
  cudaError_t e = cudaSuccess;
  const bool split = p->split && !is_f32 && map_in == kMapNone && map_out == kOutNone && ((uintptr_t)in % 16) == 0 &&
                     ((uintptr_t)out % 16) == 0;
  if (split) {
    // sparse shells: copied (out of place), then their active ring pairs filtered by the units
    // kernel; dense shells: the shell kernel over their list (both orders: a sparse shell's only
    // pass is the symmetric phi pass). The two sets of shells are disjoint, so when both have work
    // the copy (high-priority side stream) and then the units kernel (normal-priority side stream)
    // run beside the shell kernel on the caller's stream. The chunks of the host-buffer pipeline
    // (tc_set > 0) run all three on their own stream: the chunks on the pipeline's compute streams
    // overlap one another, which forking every chunk to the plan's one pair of side streams would
    // serialise.
    const int vb = var_begin, ve = var_begin + var_count;
    const int d0 = p->dense_off[(size_t)vb], d1 = p->dense_off[(size_t)ve];
    const int s0 = p->sparse_off[(size_t)vb], s1 = p->sparse_off[(size_t)ve];
    const int u0 = p->units_off[(size_t)vb], u1 = p->units_off[(size_t)ve];
    const bool copy = in != out && s1 > s0, dense_work = d1 > d0, side_work = copy || u1 > u0;
    const bool fork = dense_work && side_work && tc_set == 0;
    std::lock_guard<std::mutex> lock(p->split_mu);
    cudaStream_t s_main = (cudaStream_t)stream, aux_s = fork ? p->side : s_main;
    cudaStream_t copy_s = fork ? p->side_copy : s_main;
    int n = 0;
    if (fork) {
      e = cudaEventRecord(p->ev_fork, s_main);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(copy ? copy_s : aux_s, p->ev_fork, 0);
    }
    if (e == cudaSuccess && dense_work) {
      LaunchIO dense = io;
      dense.var_begin = 0;
      dense.var_count = p->nvars;
      dense.list = p->d_dense + d0;
      dense.nlist = d1 - d0;
      e = launch_shell(p->args2, p->precision, p->threads2, p->smem2, dense, s_main);
      ++n;
    }
    if (e == cudaSuccess && copy) {
      e = launch_copy_shells(static_cast<const double*>(in), static_cast<double*>(out), p->d_sparse + s0, s1 - s0,
                             (size_t)p->Nth * p->Nph, copy_s);
      ++n;
    }
    if (fork && copy) {
      // the units kernel overwrites rows of the copied shells: it waits for the copy (joined even
      // after an error, like the final join below)
      cudaError_t ec = cudaEventRecord(p->ev_copy, copy_s);
      if (ec == cudaSuccess) ec = cudaStreamWaitEvent(aux_s, p->ev_copy, 0);
      if (e == cudaSuccess) e = ec;
    }
    if (e == cudaSuccess && u1 > u0) {
      e = launch_units(p->args2, p->precision, p->smem_units, io, p->d_units + u0, u1 - u0, aux_s);
      ++n;
    }
    if (fork) {
      // join even after an error, so that the caller's stream (or capture) is never left forked
      cudaError_t ej = cudaEventRecord(p->ev_join, aux_s);
      if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s_main, p->ev_join, 0);
      if (e == cudaSuccess) e = ej;
    }
    if (e == cudaSuccess) p->launched += n;
  } else {
    e = !p->use_v2 ? launch_plain(*p, io, (cudaStream_t)stream)
        : p->cluster ? launch_shell_cl(p->args2, p->precision, p->threads2, p->smem2, io, (cudaStream_t)stream)
                     : launch_shell(p->args2, p->precision, p->threads2, p->smem2, io, (cudaStream_t)stream);
    if (e == cudaSuccess) p->launched += 1;
  }
  if (cur != p->device) cudaSetDevice(cur);
  return e == cudaSuccess ? SPH_OK : SPH_ECUDA;
}

namespace {
sph_status launch(sph_filter_plan p, const void* in, const void* aux, void* out, int map_in, int map_out,
                  int transpose, int is_f32, sph_stream_t stream) {
  return launch_plan(p, in, aux, out, map_in, map_out, transpose, is_f32, (cudaStream_t)stream);
}
}  // namespace
}  // namespace sph

using namespace sph;

extern "C" {

sph_status sph_filter_plan_create(sph_filter_plan* out, int Nr, int Ntheta, int Nphi, int nvars,
                                  const int* parity, const sph_cutoff_params* prm) {
  if (!out) return SPH_EINVAL;
  *out = nullptr;
  if (!parity || !prm || !prm->r || !prm->L || !prm->kind) return SPH_EINVAL;
  if (Nr < 1 || Ntheta < 1 || nvars < 1 || Nphi < 2 || (Nphi % 2) != 0) return SPH_EINVAL;
  if (!(prm->dr_min > 0) || !(prm->floor >= 0) || !std::isfinite(prm->dr_min) || !std::isfinite(prm->floor))
    return SPH_EINVAL;
  if (prm->precision != SPH_PREC_F64 && prm->precision != SPH_PREC_SPLIT_TC && prm->precision != SPH_PREC_F32X2 &&
      prm->precision != SPH_PREC_SPECTRAL)
    return SPH_EINVAL;
  bool hybrid = false;
  for (int v = 0; v < nvars; ++v) {
    if (parity[v] != 0 && parity[v] != 1) return SPH_EINVAL;
    if (prm->kind[v] < SPH_FILTER_EXP || prm->kind[v] > SPH_FILTER_HYBRID) return SPH_EINVAL;
    if (!(prm->L[v] > 0) || !std::isfinite(prm->L[v])) return SPH_EINVAL;
    hybrid |= prm->kind[v] == SPH_FILTER_HYBRID;
  }
  if (hybrid && (!(prm->eps >= 0) || !std::isfinite(prm->eps))) return SPH_EINVAL;
  // the tensor-core form builds one operator per pass and class: no per-circle switch; the spectral
  // form filters whole modes, not circles
  if (hybrid && (prm->precision == SPH_PREC_SPLIT_TC || prm->precision == SPH_PREC_SPECTRAL)) return SPH_EUNSUPPORTED;
  // the spectral form's per-mode transform pairs rows 2n and 2n + 1
  if (prm->precision == SPH_PREC_SPECTRAL && (Ntheta % 2) != 0) return SPH_EUNSUPPORTED;
  for (int i = 0; i < Nr; ++i)
    if (!(prm->r[i] >= 0) || !std::isfinite(prm->r[i])) return SPH_EINVAL;

  sph_filter_plan_s* p = new (std::nothrow) sph_filter_plan_s();
  if (!p) return SPH_ENOMEM;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return SPH_ECUDA;
  }
  p->Nr = Nr;
  p->Nth = Ntheta;
  p->Nph = Nphi;
  p->nvars = nvars;
  p->precision = prm->precision;
  p->dr_min = prm->dr_min;
  p->floor_ = prm->floor;
  p->parity.assign(parity, parity + nvars);
  p->kind.assign(prm->kind, prm->kind + nvars);
  p->L.assign(prm->L, prm->L + nvars);
  p->r.assign(prm->r, prm->r + Nr);
  p->has_hybrid = hybrid;
  // cutoff classes: distinct (kind, L); a hybrid field also needs the Gaussian class of its L
  auto class_of = [p](int kind, double L) {
    int c = 0;
    for (; c < p->ncls; ++c)
      if (p->cls_kind[(size_t)c] == kind && p->cls_L[(size_t)c] == L) break;
    if (c == p->ncls) {
      p->cls_kind.push_back(kind);
      p->cls_L.push_back(L);
      ++p->ncls;
    }
    return c;
  };
  p->var_cls.resize((size_t)nvars);
  std::vector<int> alt_cls((size_t)nvars);
  for (int v = 0; v < nvars; ++v) {
    p->var_cls[(size_t)v] = class_of(p->kind[(size_t)v], p->L[(size_t)v]);
    alt_cls[(size_t)v] = p->kind[(size_t)v] == SPH_FILTER_HYBRID ? class_of(SPH_FILTER_GAUSS, p->L[(size_t)v])
                                                                 : p->var_cls[(size_t)v];
  }
  p->h_lmax.resize((size_t)p->ncls * Nr);
  p->h_mmax.resize((size_t)p->ncls * Nr * Ntheta);
  for (int c = 0; c < p->ncls; ++c)
    for (int i = 0; i < Nr; ++i) {
      p->h_lmax[(size_t)c * Nr + i] = lmax_of(p->r[(size_t)i], p->dr_min, p->cls_L[(size_t)c], p->floor_);
      for (int j = 0; j < Ntheta; ++j)
        p->h_mmax[((size_t)c * Nr + i) * Ntheta + j] =
            mmax_of(p->r[(size_t)i], p->dr_min, p->cls_L[(size_t)c], p->floor_, j, Ntheta);
    }
  std::vector<VarInfo> vi((size_t)nvars);
  for (int v = 0; v < nvars; ++v)
    vi[(size_t)v] = VarInfo{p->parity[(size_t)v], p->kind[(size_t)v], p->var_cls[(size_t)v], alt_cls[(size_t)v]};

  sph_status st = SPH_OK;
  if (st == SPH_OK) st = upload(&p->d_lmax, p->h_lmax.data(), p->h_lmax.size());
  if (st == SPH_OK) st = upload(&p->d_mmax, p->h_mmax.data(), p->h_mmax.size());
  if (st == SPH_OK) st = upload(&p->d_var, vi.data(), vi.size());
  if (st == SPH_OK) {
    if (cudaMalloc((void**)&p->d_status, sizeof(unsigned)) != cudaSuccess) st = SPH_ENOMEM;
    else if (cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess) st = SPH_ECUDA;
  }
  if (st != SPH_OK) {
    free_plan(p);
    return st;
  }
  if (p->precision == SPH_PREC_SPLIT_TC) {
    st = tc_setup(p);
    if (st != SPH_OK) {
      free_plan(p);
      return st;
    }
    p->launches = 2;
    *out = p;
    return SPH_OK;
  }
  // the staged shell kernel when the shape fits it; otherwise the chunked FP64 kernel
  p->args2.eps = prm->eps;
  {
    int e = 0;
    const double m = std::frexp(prm->eps, &e);  // eps = m 2^e, 0.5 <= m < 1 (m = 0 for eps = 0)
    p->args2.eps_m = (float)m;
    p->args2.eps_p = e;
  }
  st = setup_v2(p);
  if (st != SPH_OK && st != SPH_EUNSUPPORTED) {
    free_plan(p);
    return st;
  }
  if (hybrid && !p->use_v2) {
    // the detector and the per-circle multipliers live in the staged shell kernels
    free_plan(p);
    return SPH_EUNSUPPORTED;
  }
  if (p->precision == SPH_PREC_SPECTRAL && (!p->use_v2 || p->cluster)) {
    // the spectral form runs in the single-CTA staged shell kernel only
    free_plan(p);
    return SPH_EUNSUPPORTED;
  }
  if (!p->use_v2) {
    if (p->precision != SPH_PREC_F64) {
      free_plan(p);
      return SPH_EUNSUPPORTED;
    }
    ShellArgs& a = p->args;
    a.Nr = Nr;
    a.Nth = Ntheta;
    a.Nph = Nphi;
    a.nvars = nvars;
    a.ldS = Nphi + 1;
    if (!factorize(2 * Ntheta, &a.f_th) || !factorize(Nphi, &a.f_ph)) {
      free_plan(p);
      return SPH_EUNSUPPORTED;
    }
    p->smem_bytes = plain_smem_bytes(a, &a.chunk_th, &a.chunk_ph);
    if (p->smem_bytes == 0) {
      free_plan(p);
      return SPH_EUNSUPPORTED;
    }
    auto tth = twiddles(2 * Ntheta);
    auto tph = twiddles(Nphi);
    st = upload(&p->d_tw_th, tth.data(), tth.size());
    if (st == SPH_OK) st = upload(&p->d_tw_ph, tph.data(), tph.size());
    if (st == SPH_OK && set_plain_smem_attr(p->smem_bytes) != cudaSuccess) st = SPH_ECUDA;
    if (st != SPH_OK) {
      free_plan(p);
      return st;
    }
    a.lmax = p->d_lmax;
    a.mmax = p->d_mmax;
    a.var = p->d_var;
    a.tw_th = p->d_tw_th;
    a.tw_ph = p->d_tw_ph;
    a.status = p->d_status;
  }
  p->launches = p->split ? 3 : 1;  // split: shell copy, dense shells, units (out of place)
  *out = p;
  return SPH_OK;
}

void sph_filter_plan_destroy(sph_filter_plan plan) {
  if (!plan) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  free_plan(plan);
  if (cur >= 0) cudaSetDevice(cur);
}

sph_status sph_filter_apply(sph_filter_plan plan, const double* in, double* out, sph_stream_t stream) {
  return launch(plan, in, nullptr, out, kMapNone, kOutNone, 0, 0, stream);
}

sph_status sph_filter_apply_adjoint(sph_filter_plan plan, const double* in, double* out, sph_stream_t stream) {
  return launch(plan, in, nullptr, out, kMapNone, kOutNone, 1, 0, stream);
}

sph_status sph_filter_apply_tanh(sph_filter_plan plan, const double* z, double* out, sph_stream_t stream) {
  return launch(plan, z, nullptr, out, kMapTanh, kOutNone, 0, 0, stream);
}

sph_status sph_filter_apply_adjoint_tanh(sph_filter_plan plan, const double* g, const double* z, double* out,
                                         sph_stream_t stream) {
  return launch(plan, g, z, out, kMapNone, kOutTanhGrad, 1, 0, stream);
}

sph_status sph_filter_apply_f32(sph_filter_plan plan, const float* in, float* out, sph_stream_t stream) {
  return launch(plan, in, nullptr, out, kMapNone, kOutNone, 0, 1, stream);
}

sph_status sph_filter_apply_adjoint_f32(sph_filter_plan plan, const float* in, float* out, sph_stream_t stream) {
  return launch(plan, in, nullptr, out, kMapNone, kOutNone, 1, 1, stream);
}

sph_status sph_filter_apply_tanh_f32(sph_filter_plan plan, const float* z, float* out, sph_stream_t stream) {
  return launch(plan, z, nullptr, out, kMapTanh, kOutNone, 0, 1, stream);
}

sph_status sph_filter_apply_adjoint_tanh_f32(sph_filter_plan plan, const float* g, const float* z, float* out,
                                             sph_stream_t stream) {
  return launch(plan, g, z, out, kMapNone, kOutTanhGrad, 1, 1, stream);
}

sph_status sph_filter_apply_host(sph_filter_plan plan, const double* host_in, double* host_out,
                                 sph_stream_t stream) {
  if (!plan || !host_in || !host_out) return SPH_EINVAL;
  const size_t field = (size_t)plan->Nr * plan->Nth * plan->Nph;  // values per field
  const size_t n = field * plan->nvars;
  if (!plan->d_stage_in) {
    if (cudaMalloc((void**)&plan->d_stage_in, sizeof(double) * n) != cudaSuccess) return SPH_ENOMEM;
    if (cudaMalloc((void**)&plan->d_stage_out, sizeof(double) * n) != cudaSuccess) {
      cudaFree(plan->d_stage_in);
      plan->d_stage_in = nullptr;
      return SPH_ENOMEM;
    }
  }
  if (plan->tc) {
    const sph_status st = tc_reserve_pipeline(plan);
    if (st != SPH_OK) return st;
  }
  if (!plan->pipe_in) {
    for (cudaStream_t* q : {&plan->pipe[0], &plan->pipe[1], &plan->pipe[2], &plan->pipe[3], &plan->pipe[4],
                            &plan->pipe[5], &plan->pipe_out, &plan->pipe_in})  // pipe_in last: the "created" mark
      if (cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess) {
        *q = nullptr;
        return SPH_ECUDA;
      }
  }
  if (!plan->pipe_end) {
    for (cudaEvent_t* e : {&plan->pipe_start, &plan->pipe_end})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
        *e = nullptr;
        return SPH_ECUDA;
      }
  }
  if ((int)plan->chunk_done.size() < plan->nvars) {  // one chunk per field at most
    for (std::vector<cudaEvent_t>* v : {&plan->chunk_in, &plan->chunk_done})
      while ((int)v->size() < plan->nvars) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SPH_ECUDA;
        v->push_back(e);
      }
  }
  // Pipeline over chunks of whole fields: the copies in run back to back on one stream, each chunk's
  // kernels on a compute stream once its copy has landed, and the copies out back to back on another
  // stream, each once its chunk's kernels are done. The staging buffers hold the whole state, so no
  // chunk waits for another's buffer: both directions of the host link stay busy from the first
  // chunk to the last, and the kernels of several chunks overlap.
  cudaStream_t s = (cudaStream_t)stream;
  // chunks of about 16 MiB: small enough that filling and draining the pipeline costs little, large
  // enough that each copy runs at the link's full rate
  const size_t field_bytes = sizeof(double) * field;
  const int chunk = (int)std::min<size_t>(plan->nvars, std::max<size_t>(1, ((16u << 20) + field_bytes / 2) / field_bytes));
  // compute streams: an FP64 chunk's kernels take about one shell's time (one partial wave of CTAs,
  // ~0.23 ms for 64 x 128 shells) while a chunk arrives every ~0.08 ms, so up to six chunks run at
  // once; the tensor-core form has three pipeline counter sets, one per stream
  constexpr int kP = sph_filter_plan_s::kPipeStreams;
  const int nstreams = plan->tc ? 3 : kP;
  if (cudaEventRecord(plan->pipe_start, s) != cudaSuccess) return SPH_ECUDA;
  if (cudaStreamWaitEvent(plan->pipe_in, plan->pipe_start, 0) != cudaSuccess) return SPH_ECUDA;
  // the first and the last chunk hold one field: the pipeline fills and drains faster
  const bool taper = chunk > 1 && plan->nvars > 2;
  int k = 0;
  for (int v0 = 0, nv = 0; v0 < plan->nvars; v0 += nv, ++k) {
    const int left = plan->nvars - v0;
    nv = (taper && (k == 0 || left == 1)) ? 1 : std::max(1, std::min(chunk, taper ? left - 1 : left));
    cudaStream_t cs = plan->pipe[k % nstreams];
    const size_t off = field * v0, cnt = field * nv;
    if (cudaMemcpyAsync(plan->d_stage_in + off, host_in + off, sizeof(double) * cnt, cudaMemcpyHostToDevice,
                        plan->pipe_in) != cudaSuccess)
      return SPH_ECUDA;
    if (cudaEventRecord(plan->chunk_in[k], plan->pipe_in) != cudaSuccess) return SPH_ECUDA;
    if (cudaStreamWaitEvent(cs, plan->chunk_in[k], 0) != cudaSuccess) return SPH_ECUDA;
    // the tensor-core form's scratch set of this stream (chunks on different streams may overlap)
    const sph_status st = launch_plan_vars(plan, plan->d_stage_in, nullptr, plan->d_stage_out, kMapNone, kOutNone, 0,
                                           0, v0, nv, cs, 1 + k % 3);
    if (st != SPH_OK) return st;
    if (cudaEventRecord(plan->chunk_done[k], cs) != cudaSuccess) return SPH_ECUDA;
    if (cudaStreamWaitEvent(plan->pipe_out, plan->chunk_done[k], 0) != cudaSuccess) return SPH_ECUDA;
    if (cudaMemcpyAsync(host_out + off, plan->d_stage_out + off, sizeof(double) * cnt, cudaMemcpyDeviceToHost,
                        plan->pipe_out) != cudaSuccess)
      return SPH_ECUDA;
  }
  // every chunk's kernels precede its copy out, and the copies out run in order: the caller's stream
  // continues after the last one
  if (cudaEventRecord(plan->pipe_end, plan->pipe_out) != cudaSuccess) return SPH_ECUDA;
  if (cudaStreamWaitEvent(s, plan->pipe_end, 0) != cudaSuccess) return SPH_ECUDA;
  return SPH_OK;
}

sph_status sph_filter_plan_sync_status(sph_filter_plan plan) {
  if (!plan) return SPH_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return SPH_ECUDA;
  unsigned h = 0;
  if (cudaMemcpy(&h, plan->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return SPH_ECUDA;
  if (h != 0 && cudaMemset(plan->d_status, 0, sizeof(unsigned)) != cudaSuccess) return SPH_ECUDA;
  return (sph_status)h;
}

long long sph_filter_plan_points(sph_filter_plan plan) {
  if (!plan) return 0;
  return (long long)plan->nvars * plan->Nr * plan->Nth * plan->Nph;
}

int sph_filter_plan_launches(sph_filter_plan plan) { return plan ? plan->launches : 0; }

long long sph_filter_plan_launch_count(sph_filter_plan plan) { return plan ? plan->launched.load() : 0; }

const char* sph_filter_status_string(sph_status s) {
  switch (s) {
    case SPH_OK: return "ok";
    case SPH_EINVAL: return "invalid argument";
    case SPH_ENOMEM: return "out of memory";
    case SPH_ECUDA: return "CUDA runtime error";
    case SPH_EUNSUPPORTED: return "unsupported configuration";
    case SPH_ETIMEOUT: return "device-side wait timed out";
    case SPH_EALIAS: return "input and output partially overlap";
    case SPH_EDEVICE: return "device-side consistency error";
  }
  return "unknown status";
}

}  // extern "C"
