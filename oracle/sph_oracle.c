/*
 * Oracle for the double FFT filter of Ji et al., "Ameliorating the CFL condition in spherical
 * coordinates: a double FFT filter method for GRMHD in dynamical spacetimes" (arXiv:2305.01537),
 * Sec. II.C "Filtering algorithms".
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct CPU statement of what the
 * filter computes. Only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * may load it. The CUDA library shares no code, header, table or helper with this file.
 *
 * Every transform here is a naive O(N^2) discrete Fourier transform with exact integer index
 * reduction ((l*q) mod N) into a cosine table; there is no FFT, no blocking and no fusion, so a
 * reader can check each step against the paper by eye.
 *
 * The file is compiled twice: with REAL = double (the oracle proper) and with REAL = long double
 * (-DORACLE_LONG_DOUBLE; 80-bit extended on x86-64, IEEE binary128 on aarch64). The second build
 * bounds the rounding error of the first. Inputs and outputs are always double.
 *
 * Layout of a state: x[v][i][j][k], v = field (variable), i = radial shell, j = theta index,
 * k = phi index (fastest). theta_j = (j + 1/2) pi / Ntheta (cell centred), phi_k = 2 pi k / Nphi.
 *
 * Readings of the paper taken here (each one is also listed in the design notes):
 *  - Order: the theta pass runs first, then the phi pass (Sec. II.C, opening paragraph).
 *  - The double covering (Sec. II.C, definition of X(x1, vartheta, phi)): for vartheta in
 *    (pi, 2 pi) the field is (-1)^a X(2 pi - vartheta, phi + pi). On the cell-centred grid the
 *    circle sample q >= Ntheta comes from theta index 2 Ntheta - 1 - q of the meridian phi + pi.
 *  - The cutoffs l_max, m_max (Sec. II.C, cutoff equations) stay real valued (no rounding); the
 *    floor "2" is a parameter whose default is 2.
 *  - Filter functions act on |l| for every signed frequency in (-N/2, N/2]; the Nyquist mode
 *    gets f(N/2).
 *  - Hybrid filter (Sec. II.C, the exponential/Gaussian switch by Jameson's shock detector): each
 *    theta circle and each phi ring of a hybrid field takes the Gaussian filter if some cell of it
 *    has sigma >= 0.95, else the exponential filter. Both detectors read the field as it enters the
 *    filter (before the theta pass). The theta detector walks the double-covered circle (the
 *    neighbours of a cell next to a pole are across the pole, with the parity sign); the phi
 *    detector walks the periodic ring. sigma is evaluated in double precision in both builds as
 *        num = |(u[i-1] + u[i+1]) - 2 u[i]|,  den = ((|u[i-1]| + |u[i+1]|) + 2 |u[i]|) + eps,
 *        fire  <=>  num / den >= 0.95,
 *    which is the paper's ratio with the two neighbours summed first (the result then does not
 *    depend on the direction in which a circle is walked). eps is the caller's parameter. The
 *    switch is nonlinear, so the transpose is not defined for hybrid fields.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_LONG_DOUBLE
typedef long double REAL;
#define RCOS cosl
#define RSIN sinl
#define REXP expl
#define RLOG logl
#define RACOS acosl
#define RFABS fabsl
#define SYM(name) oracle_ld_##name
#else
typedef double REAL;
#define RCOS cos
#define RSIN sin
#define REXP exp
#define RLOG log
#define RACOS acos
#define RFABS fabs
#define SYM(name) oracle_##name
#endif

enum { KIND_EXP = 0, KIND_GAUSS = 1, KIND_SHARP = 2, KIND_HYBRID = 3 };

/* Filter function f(l, l_max).
 *  exp:      Eq. (exp_filter):      1 for |l| <= l_max, exp(-(|l| - l_max)) above.
 *  Gaussian: Eq. (gaussian_filter): exp(log(0.9) (l / (l_max + 1))^2) for every l.
 *  sharp:    the spectrally sharp low-pass named just before Eq. (exp_filter): 1 for
 *            |l| <= l_max, 0 above. */
static REAL filter_value(int kind, REAL l, REAL lmax) {
  REAL al = RFABS(l);
  if (kind == KIND_EXP) return (al <= lmax) ? (REAL)1 : REXP(-(al - lmax));
  if (kind == KIND_GAUSS) {
    REAL t = l / (lmax + 1);
    return REXP(RLOG((REAL)0.9) * t * t);
  }
  return (al <= lmax) ? (REAL)1 : (REAL)0;
}

/* Cutoffs, Sec. II.C: l_max = max(2, 2 r / dr_min * L), m_max = max(2, 2 r / dr_min * sin(theta) * L).
 * The constant 2 of the max() is the parameter `floor_`. */
static REAL lmax_of(REAL r, REAL dr_min, REAL L, REAL floor_) {
  REAL v = 2 * r / dr_min * L;
  return v > floor_ ? v : floor_;
}
static REAL mmax_of(REAL r, REAL dr_min, REAL L, REAL floor_, REAL theta) {
  REAL v = 2 * r / dr_min * RSIN(theta) * L;
  return v > floor_ ? v : floor_;
}

/* Jameson's shock detector (Sec. II.C) on one cell with neighbours a, c: 1 if sigma >= 0.95. Always
 * double precision (the decision must not depend on the build). */
static int jameson_fires(double a, double b, double c, double eps) {
  double num = fabs((a + c) - 2.0 * b);
  double den = ((fabs(a) + fabs(c)) + 2.0 * fabs(b)) + eps;
  return num / den >= 0.95;
}

/* Detector flags of one shell x[j][k] (double input): circ[k] for the theta circles k < Nphi/2 (the
 * circle of 2 Ntheta samples joining meridians k and k + Nphi/2 over the poles with the sign), and
 * ring[j] for the phi rings. */
static void detect_shell(int Nth, int Nph, int parity, double eps, const double* x, unsigned char* circ,
                         unsigned char* ring) {
  int M = 2 * Nth, half = Nph / 2;
  double sign = parity ? -1.0 : 1.0;
  double* c = (double*)malloc(sizeof(double) * (size_t)(M > Nph ? M : Nph));
  for (int k = 0; k < half; ++k) {
    for (int q = 0; q < M; ++q)
      c[q] = q < Nth ? x[(size_t)q * Nph + k] : sign * x[(size_t)(M - 1 - q) * Nph + (k + half)];
    circ[k] = 0;
    for (int q = 0; q < M; ++q)
      if (jameson_fires(c[(q + M - 1) % M], c[q], c[(q + 1) % M], eps)) circ[k] = 1;
  }
  for (int j = 0; j < Nth; ++j) {
    const double* row = x + (size_t)j * Nph;
    ring[j] = 0;
    for (int k = 0; k < Nph; ++k)
      if (jameson_fires(row[(k + Nph - 1) % Nph], row[k], row[(k + 1) % Nph], eps)) ring[j] = 1;
  }
  free(c);
}

/* The filter function a circle or ring uses: a hybrid field's Gaussian where its detector fired,
 * else its exponential. */
static int kind_used(int kind, const unsigned char* fired, int idx) {
  if (kind != KIND_HYBRID) return kind;
  return fired[idx] ? KIND_GAUSS : KIND_EXP;
}

/* Low-pass one real sequence c[0..M-1] in place: naive DFT over the signed frequencies
 * l in (-M/2, M/2] (M even) or [-(M-1)/2, (M-1)/2] (M odd), multiply each coefficient by
 * f(|l|, cut), naive inverse DFT with 1/M, keep the real part. ctab[n] = cos(2 pi n / M),
 * stab[n] = sin(2 pi n / M). Work buffers re/im hold M entries. */
static void lowpass_sequence(int M, REAL* c, int kind, REAL cut, const REAL* ctab, const REAL* stab,
                             REAL* re, REAL* im, REAL* tmp) {
  int lo = -((M - 1) / 2), hi = M / 2; /* signed frequency range, M values */
  for (int l = lo; l <= hi; ++l) {
    int lm = ((l % M) + M) % M;
    REAL sr = 0, si = 0;
    for (int q = 0; q < M; ++q) {
      int n = (int)(((long)lm * q) % M);
      sr += c[q] * ctab[n];
      si -= c[q] * stab[n];
    }
    REAL f = filter_value(kind, (REAL)l, cut);
    re[l - lo] = sr * f;
    im[l - lo] = si * f;
  }
  for (int q = 0; q < M; ++q) {
    REAL s = 0;
    for (int l = lo; l <= hi; ++l) {
      int lm = ((l % M) + M) % M;
      int n = (int)(((long)lm * q) % M);
      /* real part of (re + i im) (cos + i sin) */
      s += re[l - lo] * ctab[n] - im[l - lo] * stab[n];
    }
    tmp[q] = s / (REAL)M;
  }
  memcpy(c, tmp, sizeof(REAL) * (size_t)M);
}

static void make_tables(int M, REAL* ctab, REAL* stab) {
  REAL twopi = 2 * RACOS((REAL)-1);
  for (int n = 0; n < M; ++n) {
    ctab[n] = RCOS(twopi * (REAL)n / (REAL)M);
    stab[n] = RSIN(twopi * (REAL)n / (REAL)M);
  }
}

/* theta pass on one shell s[j][k] (Ntheta x Nphi), in place (Sec. II.C, first filter equation and
 * the double-covering definition). For each meridian pair (k, k + Nphi/2), k < Nphi/2, build the
 * circle of 2 Ntheta samples, low-pass it with f(|l|, l_max) and scatter back with the sign.
 * circ: detector flags of a hybrid field (unused otherwise). */
static void theta_pass_shell(int Nth, int Nph, int parity, int kind, const unsigned char* circ, REAL lmax,
                             REAL* s) {
  int M = 2 * Nth, half = Nph / 2;
  REAL sign = parity ? (REAL)-1 : (REAL)1;
  REAL* buf = (REAL*)malloc(sizeof(REAL) * (size_t)M * 6);
  REAL *c = buf, *ctab = buf + M, *stab = buf + 2 * M, *re = buf + 3 * M, *im = buf + 4 * M,
       *tmp = buf + 5 * M;
  make_tables(M, ctab, stab);
  for (int k = 0; k < half; ++k) {
    for (int q = 0; q < M; ++q) {
      if (q < Nth) c[q] = s[(size_t)q * Nph + k];
      else c[q] = sign * s[(size_t)(M - 1 - q) * Nph + (k + half)];
    }
    lowpass_sequence(M, c, kind_used(kind, circ, k), lmax, ctab, stab, re, im, tmp);
    for (int j = 0; j < Nth; ++j) {
      s[(size_t)j * Nph + k] = c[j];
      s[(size_t)j * Nph + (k + half)] = sign * c[M - 1 - j];
    }
  }
  free(buf);
}

/* phi pass on one shell (Sec. II.C, second filter equation): each ring j is low-passed with
 * f(|m|, m_max(r, theta_j)). ring: detector flags of a hybrid field (unused otherwise). */
static void phi_pass_shell(int Nth, int Nph, int kind, const unsigned char* ring, REAL r, REAL dr_min, REAL L,
                           REAL floor_, REAL* s) {
  int M = Nph;
  REAL pi = RACOS((REAL)-1);
  REAL* buf = (REAL*)malloc(sizeof(REAL) * (size_t)M * 6);
  REAL *c = buf, *ctab = buf + M, *stab = buf + 2 * M, *re = buf + 3 * M, *im = buf + 4 * M,
       *tmp = buf + 5 * M;
  make_tables(M, ctab, stab);
  for (int j = 0; j < Nth; ++j) {
    REAL theta = ((REAL)j + (REAL)0.5) * pi / (REAL)Nth;
    REAL mmax = mmax_of(r, dr_min, L, floor_, theta);
    for (int k = 0; k < M; ++k) c[k] = s[(size_t)j * Nph + k];
    lowpass_sequence(M, c, kind_used(kind, ring, j), mmax, ctab, stab, re, im, tmp);
    for (int k = 0; k < M; ++k) s[(size_t)j * Nph + k] = c[k];
  }
  free(buf);
}

static int check_args(int Nr, int Nth, int Nph, int nvars, const int* parity, const int* kind,
                      const double* L, const double* r, double dr_min, double floor_, double eps) {
  if (Nr < 1 || Nth < 1 || Nph < 2 || (Nph % 2) != 0 || nvars < 1) return 1;
  if (!parity || !kind || !L || !r || !(dr_min > 0) || !(floor_ >= 0) || !(eps >= 0)) return 1;
  for (int v = 0; v < nvars; ++v) {
    if (parity[v] != 0 && parity[v] != 1) return 1;
    if (kind[v] < 0 || kind[v] > 3) return 1;
    if (!(L[v] > 0)) return 1;
  }
  for (int i = 0; i < Nr; ++i)
    if (!(r[i] >= 0)) return 1;
  return 0;
}

/* which: bit 0 = theta pass, bit 1 = phi pass; order 0 = theta then phi (the filter),
 * order 1 = phi then theta (its transpose, since each pass is a real symmetric operator; not
 * defined for hybrid fields). */
static int run(int Nr, int Nth, int Nph, int nvars, const int* parity, const int* kind,
               const double* L, const double* r, double dr_min, double floor_, double eps,
               const double* in, double* out, int which, int order) {
  if (check_args(Nr, Nth, Nph, nvars, parity, kind, L, r, dr_min, floor_, eps)) return 1;
  if (order != 0)
    for (int v = 0; v < nvars; ++v)
      if (kind[v] == KIND_HYBRID) return 1;
  long nshell = (long)nvars * Nr;
  size_t npts = (size_t)Nth * Nph;
#pragma omp parallel for schedule(dynamic, 1)
  for (long sidx = 0; sidx < nshell; ++sidx) {
    int v = (int)(sidx / Nr), i = (int)(sidx % Nr);
    REAL* s = (REAL*)malloc(sizeof(REAL) * npts);
    const double* src = in + (size_t)sidx * npts;
    for (size_t p = 0; p < npts; ++p) s[p] = (REAL)src[p];
    unsigned char* circ = (unsigned char*)calloc((size_t)(Nph / 2 + Nth), 1);
    unsigned char* ring = circ + Nph / 2;
    if (kind[v] == KIND_HYBRID) detect_shell(Nth, Nph, parity[v], eps, src, circ, ring);
    REAL lmax = lmax_of((REAL)r[i], (REAL)dr_min, (REAL)L[v], (REAL)floor_);
    for (int step = 0; step < 2; ++step) {
      int pass = (order == 0) ? step : 1 - step; /* 0 = theta, 1 = phi */
      if (pass == 0 && (which & 1)) theta_pass_shell(Nth, Nph, parity[v], kind[v], circ, lmax, s);
      if (pass == 1 && (which & 2))
        phi_pass_shell(Nth, Nph, kind[v], ring, (REAL)r[i], (REAL)dr_min, (REAL)L[v], (REAL)floor_, s);
    }
    double* dst = out + (size_t)sidx * npts;
    for (size_t p = 0; p < npts; ++p) dst[p] = (double)s[p];
    free(circ);
    free(s);
  }
  return 0;
}

/* ---- exported entry points (return 0 on success, 1 on invalid arguments) ----
 * eps: the detector's epsilon for hybrid fields (kind 3), >= 0. */

/* The double filter: theta pass, then phi pass. */
int SYM(filter)(int Nr, int Nth, int Nph, int nvars, const int* parity, const int* kind,
                const double* L, const double* r, double dr_min, double floor_, double eps,
                const double* in, double* out) {
  return run(Nr, Nth, Nph, nvars, parity, kind, L, r, dr_min, floor_, eps, in, out, 3, 0);
}

/* Transpose of the double filter: phi pass, then theta pass (rejects hybrid fields). */
int SYM(filter_T)(int Nr, int Nth, int Nph, int nvars, const int* parity, const int* kind,
                  const double* L, const double* r, double dr_min, double floor_, double eps,
                  const double* in, double* out) {
  return run(Nr, Nth, Nph, nvars, parity, kind, L, r, dr_min, floor_, eps, in, out, 3, 1);
}

/* One pass alone: which = 1 theta pass only, 2 phi pass only. Hybrid fields detect on the input. */
int SYM(single_pass)(int Nr, int Nth, int Nph, int nvars, const int* parity, const int* kind,
                     const double* L, const double* r, double dr_min, double floor_, double eps,
                     const double* in, double* out, int which) {
  if (which != 1 && which != 2) return 1;
  return run(Nr, Nth, Nph, nvars, parity, kind, L, r, dr_min, floor_, eps, in, out, which, 0);
}

/* Detector flags of one shell [Ntheta][Nphi]: circ[Nphi/2] (theta circles), ring[Ntheta] (phi rings). */
int SYM(detect)(int Nth, int Nph, int parity, double eps, const double* shell, unsigned char* circ,
                unsigned char* ring) {
  if (Nth < 1 || Nph < 2 || (Nph % 2) != 0 || (parity != 0 && parity != 1) || !(eps >= 0)) return 1;
  detect_shell(Nth, Nph, parity, eps, shell, circ, ring);
  return 0;
}

/* sigma >= 0.95 for one cell (1) or not (0). */
int SYM(jameson_fires)(double a, double b, double c, double eps) { return jameson_fires(a, b, c, eps); }

double SYM(filter_value)(int kind, double l, double lmax) {
  return (double)filter_value(kind, (REAL)l, (REAL)lmax);
}
double SYM(lmax)(double r, double dr_min, double L, double floor_) {
  return (double)lmax_of((REAL)r, (REAL)dr_min, (REAL)L, (REAL)floor_);
}
double SYM(mmax)(double r, double dr_min, double L, double floor_, int j, int Nth) {
  REAL theta = ((REAL)j + (REAL)0.5) * RACOS((REAL)-1) / (REAL)Nth;
  return (double)mmax_of((REAL)r, (REAL)dr_min, (REAL)L, (REAL)floor_, theta);
}

int SYM(max_threads)(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void SYM(set_threads)(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
