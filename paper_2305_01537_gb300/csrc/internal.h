// Internal declarations shared by the CUDA translation units of the library (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/sph_filter.h"

namespace sph {

constexpr int kMaxStages = 12;   // radix stages of one FFT length
constexpr int kThreads = 256;    // threads per CTA of the shell kernels

// Mixed-radix factorisation of an FFT length, radices in the order the stages run.
struct Factors {
  int n = 0;
  int nst = 0;
  int radix[kMaxStages] = {};
};

// Per-field description the kernels read: parity a, filter kind, cutoff-class index.
struct VarInfo {
  int parity;
  int kind;
  int cls;
  int pad;
};

// Everything a shell kernel needs, passed by value.
struct ShellArgs {
  int Nr, Nth, Nph, nvars;
  int ldS;            // row stride (doubles) of the staged shell in shared memory
  int chunk_th;       // complex sequences per theta FFT batch
  int chunk_ph;       // complex sequences per phi FFT batch
  Factors f_th;       // factors of 2 Ntheta
  Factors f_ph;       // factors of Nphi
  const double* lmax;     // [ncls][Nr]
  const double* mmax;     // [ncls][Nr][Nth]
  const VarInfo* var;     // [nvars]
  const double2* tw_th;   // [2 Nth]  exp(-2 pi i n / (2 Nth))
  const double2* tw_ph;   // [Nph]    exp(-2 pi i n / Nph)
  unsigned* status;       // device error word (0 = ok)
};

// Pointwise maps fused at the load or the store of a shell.
enum MapIn { kMapNone = 0, kMapTanh = 1 };
enum MapOut { kOutNone = 0, kOutTanhGrad = 1 };

struct LaunchIO {
  const void* in;     // state read by the filter
  const void* aux;    // z for the tanh-gradient output map (else null)
  void* out;
  int map_in;
  int map_out;
  int transpose;      // 0: theta then phi; 1: phi then theta
  int is_f32;         // 0: FP64 I/O, 1: FP32 I/O
};

}  // namespace sph

struct sph_filter_plan_s {
  int device = 0;
  int Nr = 0, Nth = 0, Nph = 0, nvars = 0, precision = 0;
  double dr_min = 1.0, floor_ = 2.0;
  std::vector<int> parity, kind, var_cls;
  std::vector<double> L, r;
  int ncls = 0;
  std::vector<int> cls_kind;
  std::vector<double> cls_L;
  std::vector<double> h_lmax, h_mmax;

  sph::ShellArgs args{};
  size_t smem_bytes = 0;
  int launches = 1;

  double* d_lmax = nullptr;
  double* d_mmax = nullptr;
  sph::VarInfo* d_var = nullptr;
  double2* d_tw_th = nullptr;
  double2* d_tw_ph = nullptr;
  unsigned* d_status = nullptr;

  // staging buffers of sph_filter_apply_host (allocated on first use)
  double* d_stage_in = nullptr;
  double* d_stage_out = nullptr;
};

namespace sph {
// Shared-memory bytes the plain shell kernel needs for this plan's shape (0 if it cannot fit).
size_t plain_smem_bytes(const ShellArgs& a, int* chunk_th, int* chunk_ph);
// Enqueue the plain FP64 shell kernel.
cudaError_t launch_plain(const sph_filter_plan_s& p, const LaunchIO& io, cudaStream_t s);
// Largest dynamic shared memory a CTA may use on this device.
int max_smem_optin(int device);
}  // namespace sph
