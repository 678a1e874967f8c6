// Plan-time description of the split-precision tensor-core form (tc.cu): how a pass of length L
// is split into symmetry blocks, and the per-block GEMMs the kernel runs. Internal header.
#pragma once

#include <cstdint>
#include <vector>

namespace sph {
namespace tcx {

constexpr int kV = 64;        // vectors per tile
constexpr int kM = 128;       // GEMM rows (two halves of 64)
constexpr int kS = 6;         // base-256 digits per operand
constexpr int kMaxG = 8;      // GEMMs per pass
constexpr int kMaxL = 256;    // longest vector
constexpr int kMaxMap = 2048; // int16 entries of the index maps of one pass

// One block GEMM pair of a pass (forward transform to the block's Fourier modes, then back).
// Row half h (rows 64h .. 64h + 63) holds the block's coordinates of the 64 vectors of a tile:
// for a level, h = 0 is the reflection-even copy and h = 1 the reflection-odd copy (same
// operator); for the base, h = 0 is the reflection-even half and h = 1 the odd half, either side by
// side in one GEMM ("concat": half h uses output columns [h K, (h + 1) K)) or as two GEMMs that use
// rows 0 .. 63 only (rows2 = 0).
struct GemmDesc {
  int Kc;           // coordinates per half, padded to a multiple of 16 (forward K, inverse N per half)
  int Km;           // modes per half, padded to a multiple of 16 (forward N per half, inverse K)
  int concat;       // halves side by side in the output columns
  int rows2;        // rows 64 .. 127 carry data
  int Pb;           // operator fixed-point bits: entry = digits * 2^-Pb (45 .. 48)
  int rin;          // right shift that brings the block's coordinates (|c| < 2^(F + growth)) to 46 bits
  uint32_t fwd_off; // byte offset of the forward operator [kS][Nf][Kc] in the pass's operator blob
  uint32_t inv_off; // byte offset of the inverse operator [kS][Ni][Km]
  uint32_t fwd_bytes, inv_bytes;
  int kin_off;      // int16 map kin[2][Kc]: store index of coordinate k of half h (-1: padding)
  int mode_off;     // int16 map mode[2][Km]: Fourier mode m of output/input j of half h (-1: padding)
  // the same maps in affine form (checked at plan creation): for k < cnt[h], store index
  // ka[h] + ks[h] k and mode ma[h] + ms[h] k; cnt[h] = 0 for a half without data
  int cnt[2], ka[2], ks[2], ma[2], ms[2];
};

struct PassDesc {
  int L;            // vector length
  int nl;           // symmetry levels (each halves the vector: T-odd part split into two equal copies)
  int nb;           // base length after the levels (split into its reflection-even and -odd halves)
  int F;            // fractional bits of the fixed-point store: |x| < 2^ex is held as x 2^(F - ex)
  int ngemm;
  GemmDesc g[kMaxG];
  int KA, NA;       // largest K and N of any GEMM (tensor-memory layout)
  int tmem_cols;    // allocation (power of two <= 512)
  int threads;      // 128 x (warps per tensor-memory lane quarter)
  uint32_t op_max;  // largest single operator (bytes): the shared-memory operator buffer
  int nmap;         // int16 map entries
};

// The orthonormal mode basis of a GEMM's blocks: U[h][j][k] is basis vector j (Fourier mode
// modes[h][j]) over the block's coordinates k, for row half h (a level's halves share U[0]; a base
// GEMM without a second half leaves h = 1 empty).
struct GemmBasis {
  std::vector<int> modes[2];
  std::vector<std::vector<long double>> U[2];
};

// Builds the pass description, the operator blob (BF16 digit slices in the kernel's shared-memory
// layout) and the int16 index maps for vectors of length L, and (if basis is not null) the bases.
// Returns false if L is not supported.
bool build_pass_desc(int L, PassDesc* d, std::vector<uint16_t>* ops, std::vector<int16_t>* maps,
                     std::vector<GemmBasis>* basis = nullptr);

// The direct operator of GEMM g for the multipliers mu[m] (m = 0 .. L/2): the block matrix
// K = U^T diag(mu) U (rows: output coordinates, (concat ? 2 : 1) Kc of them; columns: input
// coordinates, Kc), appended to ops as digit slices at scale 2^Pb. Returns its byte offset.
uint32_t append_direct_op(const PassDesc& d, int g, const GemmBasis& b, const long double* mu,
                          std::vector<uint16_t>* ops, int* Pb);

// Offset (elements) of (row, k) in a ROWS x K operand stored K-major without swizzle: 8-row x
// 8-element core matrices of 128 contiguous bytes; the next core matrix along K is 128 bytes on,
// the next group of 8 rows (K / 8) * 128 bytes on.
inline uint32_t kmaj_elem(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K / 8) * 64 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7));
}

}  // namespace tcx
}  // namespace sph
