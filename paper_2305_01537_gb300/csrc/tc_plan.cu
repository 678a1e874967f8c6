// Plan-time construction of the split-precision tensor-core form's symmetry blocks (host code).
//
// Each pass of the double filter (Sec. II.C) applies, to every vector c of length L (a doubled
// great circle, L = 2 Ntheta, or a ring, L = Nphi), the real symmetric circulant H = I - M that
// removes the filtered part of each Fourier mode m by the factor mu_m = 1 - f(|m|, cutoff). H
// commutes with the half-length shift T: k -> k + L/2 and with the reflection R: k -> L - 1 - k
// (every shift and every reflection of the periodic index), so it is block diagonal in coordinates
// adapted to them. A "level" takes the current vector v of length n (n divisible by 4) to
//   e_k = v_k + v_{k + n/2}                       (T-even part, length n/2: the next level's vector)
//   z_k = v_k - v_{k + n/2}                       (T-odd part, length n/2)
//   a_p = z_p - z_{n/2 - 1 - p},  b_p = z_{n/4 - 1 - p} + z_{n/4 + p},   p < n/4
// The T-odd part holds the modes m with m / 2^(level - 1) odd; a (the R-even half) carries their
// cosine-like components and b (the R-odd half, index reversed) their sine-like ones, and H acts on
// a and on b by the same n/4 x n/4 matrix (the quarter shift maps one half onto the other and
// commutes with H). After the levels, the remaining T-even vector of length nb is split by R into
// its even half (v_p + v_{nb - 1 - p}) and its odd half (v_p - v_{nb - 1 - p}). Every block is
// diagonalised by an orthonormal set of restricted Fourier modes u_m, so on a block
//   W = U^T diag(mu) U w,
// which the kernel runs as two GEMMs (U, then U^T) with the per-vector multipliers in between.
// The blocks, their modes and the bases u_m are found numerically here, from the Fourier mode
// vectors themselves, in extended precision, and checked (each mode lands in exactly one block;
// the two halves of a level have the same modes and the same basis up to sign).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tc2_host.h"

namespace sph {
namespace tcx {
namespace {

int pad16(int n) { return (n + 15) / 16 * 16; }

// The level lengths' count and the base length for vectors of length L.
void plan_levels(int L, int* nl, int* nb) {
  int n = L, l = 0;
  while (n % 4 == 0 && n / 4 >= 16 && n / 2 >= 32) {
    ++l;
    n /= 2;
  }
  *nl = l;
  *nb = n;
}

// Forward coordinates in the kernel's in-place layout (levels, then the base split).
void forward_coords(std::vector<long double>& s, int L, int nl, int nb) {
  int n = L;
  for (int l = 0; l < nl; ++l, n /= 2) {
    const int q = n / 4;
    for (int p = 0; p < q; ++p) {
      const long double vp = s[p], vq = s[p + n / 2], vr = s[n / 2 - 1 - p], vs = s[n - 1 - p];
      const long double e0 = vp + vq, z0 = vp - vq, e1 = vr + vs, z1 = vr - vs;
      s[p] = e0;
      s[n / 2 - 1 - p] = e1;
      s[n / 2 + p] = z0 - z1;
      s[n - 1 - p] = z0 + z1;
    }
  }
  for (int p = 0; p < nb / 2; ++p) {
    const long double a = s[p], b = s[nb - 1 - p];
    s[p] = a + b;
    s[nb - 1 - p] = a - b;
  }
}

struct Block {
  std::vector<int> idx;                       // store index of coordinate k
  std::vector<int> modes;                     // Fourier mode of basis vector j
  std::vector<std::vector<long double>> u;    // orthonormal basis vectors (over the block's coordinates)
};

uint16_t bf16_of_digit(int d) {
  const float f = (float)d;  // |d| <= 128: exact in BF16
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

// Six balanced base-256 digits of the integer t (|t| < 2^46), most significant first.
void digits6(long long t, int d[kS]) {
  const unsigned long long tb = (unsigned long long)(t + 0x808080808080LL);
  for (int a = 0; a < kS; ++a) d[a] = (int)((tb >> (8 * (kS - 1 - a))) & 0xFF) - 128;
}

// Appends a ROWS x K operator (entries e(n, k), zero outside) as kS digit slices at scale 2^Pb.
template <class E>
uint32_t append_op(std::vector<uint16_t>* ops, int rows, int K, int Pb, E e) {
  const uint32_t off = (uint32_t)(ops->size() * 2);
  const size_t slice = (size_t)rows * K;
  ops->resize(ops->size() + kS * slice, 0);
  uint16_t* base = ops->data() + off / 2;
  for (int n = 0; n < rows; ++n)
    for (int k = 0; k < K; ++k) {
      const long double v = e(n, k);
      if (v == 0.0L) continue;
      int d[kS];
      digits6(llroundl(ldexpl(v, Pb)), d);
      for (int a = 0; a < kS; ++a) base[a * slice + kmaj_elem(n, k, K)] = bf16_of_digit(d[a]);
    }
  return off;
}

int op_bits(const std::vector<std::vector<long double>>& u) {
  long double mx = 0;
  for (const auto& r : u)
    for (long double v : r) mx = std::max(mx, fabsl(v));
  if (mx <= 0) return 48;
  const int pb = (int)floorl(45.999L - log2l(mx));
  return std::min(48, pb);
}

}  // namespace

bool build_pass_desc(int L, PassDesc* d, std::vector<uint16_t>* ops, std::vector<int16_t>* maps,
                     std::vector<GemmBasis>* basis) {
  if (L < 2 || L % 2 != 0 || L > kMaxL) return false;
  *d = PassDesc{};
  ops->clear();
  maps->clear();
  if (basis) basis->clear();
  int nl = 0, nb = 0;
  plan_levels(L, &nl, &nb);
  d->L = L;
  d->nl = nl;
  d->nb = nb;
  d->F = 56 - (nl + 1);
  // blocks: level l -> (2l: R-even half a, 2l + 1: R-odd half b); base -> (2 nl: even, 2 nl + 1: odd)
  const int nblk = 2 * nl + 2;
  std::vector<Block> blk((size_t)nblk);
  {
    int n = L;
    for (int l = 0; l < nl; ++l, n /= 2) {
      const int q = n / 4;
      for (int p = 0; p < q; ++p) {
        blk[(size_t)2 * l].idx.push_back(n / 2 + p);
        blk[(size_t)2 * l + 1].idx.push_back(n - q + p);
      }
    }
    for (int p = 0; p < nb / 2; ++p) {
      blk[(size_t)2 * nl].idx.push_back(p);
      blk[(size_t)2 * nl + 1].idx.push_back(nb - 1 - p);
    }
  }
  // Fourier mode vectors cos / sin (2 pi m (k + 1/2) / L) (the R-even / R-odd real modes)
  const long double pi = acosl(-1.0L);
  std::vector<long double> s((size_t)L);
  for (int m = 0; m <= L / 2; ++m)
    for (int kind = 0; kind < 2; ++kind) {
      bool nonzero = false;
      for (int k = 0; k < L; ++k) {
        const long long num = ((long long)m * (2 * k + 1)) % (2LL * L);
        const long double ang = pi * (long double)num / (long double)L;
        s[(size_t)k] = kind == 0 ? cosl(ang) : sinl(ang);
        nonzero |= fabsl(s[(size_t)k]) > 1e-9L;
      }
      if (!nonzero) continue;
      forward_coords(s, L, nl, nb);
      long double total = 0, best = -1;
      int bi = -1;
      for (int b = 0; b < nblk; ++b) {
        long double nrm = 0;
        for (int i : blk[(size_t)b].idx) nrm += s[(size_t)i] * s[(size_t)i];
        total += nrm;
        if (nrm > best) {
          best = nrm;
          bi = b;
        }
      }
      if (bi < 0 || best <= 0 || total - best > 1e-20L * total) return false;  // not in a single block
      const long double inv = 1.0L / sqrtl(best);
      std::vector<long double> u;
      for (int i : blk[(size_t)bi].idx) u.push_back(s[(size_t)i] * inv);
      // sign convention: largest entry positive
      size_t am = 0;
      for (size_t i = 1; i < u.size(); ++i)
        if (fabsl(u[i]) > fabsl(u[am])) am = i;
      if (u[am] < 0)
        for (auto& v : u) v = -v;
      blk[(size_t)bi].modes.push_back(m);
      blk[(size_t)bi].u.push_back(u);
    }
  for (const Block& b : blk)
    if (b.modes.size() != b.idx.size()) return false;
  // the two halves of a level: same modes, same basis up to sign
  for (int l = 0; l < nl; ++l) {
    const Block &a = blk[(size_t)2 * l], &b = blk[(size_t)2 * l + 1];
    if (a.modes != b.modes) return false;
    for (size_t j = 0; j < a.u.size(); ++j)
      for (size_t k = 0; k < a.u[j].size(); ++k)
        if (fabsl(fabsl(a.u[j][k]) - fabsl(b.u[j][k])) > 1e-15L) return false;
  }
  auto add_map = [&](const std::vector<int>& h0, const std::vector<int>& h1, int width) {
    const int off = (int)maps->size();
    for (int h = 0; h < 2; ++h)
      for (int k = 0; k < width; ++k) {
        const std::vector<int>& src = h == 0 ? h0 : h1;
        maps->push_back((int16_t)(k < (int)src.size() ? src[(size_t)k] : -1));
      }
    return off;
  };
  const std::vector<int> none;
  // level GEMMs: both halves through the R-even half's basis
  for (int l = 0; l < nl; ++l) {
    const Block &a = blk[(size_t)2 * l], &b = blk[(size_t)2 * l + 1];
    GemmDesc& g = d->g[d->ngemm++];
    const int q = (int)a.idx.size();
    g.Kc = g.Km = pad16(q);
    g.concat = 0;
    g.rows2 = 1;
    g.Pb = op_bits(a.u);
    g.rin = d->F + (l + 2) - 46;  // level-l coordinates are sums of 2^(l + 2) stored values
    g.fwd_off = append_op(ops, g.Km, g.Kc, g.Pb, [&](int j, int k) {
      return (j < q && k < q) ? a.u[(size_t)j][(size_t)k] : 0.0L;
    });
    g.fwd_bytes = (uint32_t)(kS * g.Km * g.Kc * 2);
    g.inv_off = append_op(ops, g.Kc, g.Km, g.Pb, [&](int k, int j) {
      return (j < q && k < q) ? a.u[(size_t)j][(size_t)k] : 0.0L;
    });
    g.inv_bytes = (uint32_t)(kS * g.Kc * g.Km * 2);
    g.kin_off = add_map(a.idx, b.idx, g.Kc);
    g.mode_off = add_map(a.modes, b.modes, g.Km);
    if (basis) {
      GemmBasis gb;
      gb.modes[0] = a.modes;
      gb.U[0] = a.u;
      gb.modes[1] = b.modes;
      gb.U[1] = b.u;
      basis->push_back(gb);
    }
  }
  // base: the even and odd halves, side by side in one GEMM if that fits the same tensor memory
  {
    const Block &e = blk[(size_t)2 * nl], &o = blk[(size_t)2 * nl + 1];
    const int hcnt = (int)e.idx.size();
    const int Kb = pad16(hcnt);
    int KA = Kb, NA = Kb;
    for (int i = 0; i < d->ngemm; ++i) {
      KA = std::max(KA, std::max(d->g[i].Kc, d->g[i].Km));
      NA = std::max(NA, std::max(d->g[i].Kc, d->g[i].Km));
    }
    auto cols = [](int KA_, int NA_) {
      int c = 32;
      while (c < 3 * KA_ + 5 * NA_) c *= 2;
      return c;
    };
    // side by side unless that needs more tensor memory than 256 columns or than the separate form
    const int c_with = cols(KA, std::max(NA, 2 * Kb));
    const bool concat = c_with <= std::max(cols(KA, NA), 256) && c_with <= 512;
    std::vector<std::vector<long double>> both = e.u;
    both.insert(both.end(), o.u.begin(), o.u.end());
    const int Pb = op_bits(both);
    if (concat) {
      GemmDesc& g = d->g[d->ngemm++];
      g.Kc = g.Km = Kb;
      g.concat = 1;
      g.rows2 = 1;
      g.Pb = Pb;
      g.rin = d->F + (nl + 1) - 46;  // base coordinates are sums of 2^(nl + 1) stored values
      g.fwd_off = append_op(ops, 2 * Kb, Kb, Pb, [&](int n, int k) {
        const Block& B = n < Kb ? e : o;
        const int j = n % Kb;
        return (j < hcnt && k < hcnt) ? B.u[(size_t)j][(size_t)k] : 0.0L;
      });
      g.fwd_bytes = (uint32_t)(kS * 2 * Kb * Kb * 2);
      g.inv_off = append_op(ops, 2 * Kb, Kb, Pb, [&](int n, int j) {
        const Block& B = n < Kb ? e : o;
        const int k = n % Kb;
        return (j < hcnt && k < hcnt) ? B.u[(size_t)j][(size_t)k] : 0.0L;
      });
      g.inv_bytes = g.fwd_bytes;
      g.kin_off = add_map(e.idx, o.idx, Kb);
      g.mode_off = add_map(e.modes, o.modes, Kb);
      if (basis) {
        GemmBasis gb;
        gb.modes[0] = e.modes;
        gb.U[0] = e.u;
        gb.modes[1] = o.modes;
        gb.U[1] = o.u;
        basis->push_back(gb);
      }
    } else {
      for (int half = 0; half < 2; ++half) {
        const Block& B = half == 0 ? e : o;
        GemmDesc& g = d->g[d->ngemm++];
        g.Kc = g.Km = Kb;
        g.concat = 0;
        g.rows2 = 0;
        g.Pb = op_bits(B.u);
        g.rin = d->F + (nl + 1) - 46;
        g.fwd_off = append_op(ops, Kb, Kb, g.Pb, [&](int j, int k) {
          return (j < hcnt && k < hcnt) ? B.u[(size_t)j][(size_t)k] : 0.0L;
        });
        g.fwd_bytes = (uint32_t)(kS * Kb * Kb * 2);
        g.inv_off = append_op(ops, Kb, Kb, g.Pb, [&](int k, int j) {
          return (j < hcnt && k < hcnt) ? B.u[(size_t)j][(size_t)k] : 0.0L;
        });
        g.inv_bytes = g.fwd_bytes;
        g.kin_off = add_map(B.idx, none, Kb);
        g.mode_off = add_map(B.modes, none, Kb);
        if (basis) {
          GemmBasis gb;
          gb.modes[0] = B.modes;
          gb.U[0] = B.u;
          basis->push_back(gb);
        }
      }
    }
  }
  // affine forms of the index maps (the kernel computes indices instead of reading the maps)
  for (int i = 0; i < d->ngemm; ++i) {
    GemmDesc& g = d->g[i];
    for (int h = 0; h < 2; ++h) {
      const int16_t* kin = maps->data() + g.kin_off + h * g.Kc;
      const int16_t* mode = maps->data() + g.mode_off + h * g.Km;
      int n = 0;
      while (n < g.Kc && kin[n] >= 0) ++n;
      g.cnt[h] = n;
      g.ka[h] = n > 0 ? kin[0] : 0;
      g.ks[h] = n > 1 ? kin[1] - kin[0] : 1;
      g.ma[h] = n > 0 ? mode[0] : 0;
      g.ms[h] = n > 1 ? mode[1] - mode[0] : 1;
      for (int k = 0; k < g.Kc; ++k)
        if (k < n ? kin[k] != g.ka[h] + g.ks[h] * k : kin[k] >= 0) return false;
      for (int k = 0; k < g.Km; ++k)
        if (k < n ? mode[k] != g.ma[h] + g.ms[h] * k : mode[k] >= 0) return false;
    }
  }
  d->KA = 16;
  d->NA = 16;
  d->op_max = 0;
  for (int i = 0; i < d->ngemm; ++i) {
    const GemmDesc& g = d->g[i];
    d->KA = std::max(d->KA, std::max(g.Kc, g.Km));
    const int nf = g.concat ? 2 * g.Km : g.Km, ni = g.concat ? 2 * g.Kc : g.Kc;
    d->NA = std::max(d->NA, std::max(nf, ni));
    d->op_max = std::max(d->op_max, std::max(g.fwd_bytes, g.inv_bytes));
  }
  int cols = 32;
  while (cols < 3 * d->KA + 5 * d->NA) cols *= 2;
  if (cols > 512) return false;
  d->tmem_cols = cols;
  d->threads = d->KA >= 64 ? 512 : 256;
  // the mid step holds at most 3 chunks of 8 modes per thread (threads / 128 threads share a row)
  if (d->KA / 8 > 3 * (d->threads / 128)) return false;
  d->nmap = (int)maps->size();
  if (d->nmap > kMaxMap) return false;
  return true;
}

uint32_t append_direct_op(const PassDesc& d, int gi, const GemmBasis& b, const long double* mu,
                          std::vector<uint16_t>* ops, int* Pb) {
  const GemmDesc& g = d.g[gi];
  const int halves = g.concat ? 2 : 1;
  const int rows = halves * g.Kc;
  std::vector<std::vector<long double>> K((size_t)rows, std::vector<long double>((size_t)g.Kc, 0.0L));
  long double mx = 0;
  for (int h = 0; h < halves; ++h) {
    // a level's second half uses the first half's operator (the two are equal)
    const std::vector<std::vector<long double>>& U = (g.concat && h == 1) ? b.U[1] : b.U[0];
    const std::vector<int>& modes = (g.concat && h == 1) ? b.modes[1] : b.modes[0];
    const int n = (int)U.size();
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        long double s = 0;
        for (int j = 0; j < n; ++j) s += mu[modes[(size_t)j]] * U[(size_t)j][(size_t)p] * U[(size_t)j][(size_t)q];
        K[(size_t)(h * g.Kc + p)][(size_t)q] = s;
        mx = std::max(mx, fabsl(s));
      }
  }
  *Pb = mx > 0 ? std::min(48, (int)floorl(45.999L - log2l(mx))) : 48;
  return append_op(ops, rows, g.Kc, *Pb, [&](int n, int k) { return K[(size_t)n][(size_t)k]; });
}

}  // namespace tcx
}  // namespace sph
