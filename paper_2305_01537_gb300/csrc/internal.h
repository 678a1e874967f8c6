// Internal declarations shared by the CUDA translation units of the library (not installed).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/sph_filter.h"

namespace sph {

constexpr int kMaxStages = 12;   // radix stages of one FFT length
constexpr int kThreads = 256;    // threads per CTA of the chunked FP64 kernel

// Mixed-radix factorisation of an FFT length, radices in the order the stages run.
struct Factors {
  int n = 0;
  int nst = 0;
  int radix[kMaxStages] = {};
};

// Per-field description the kernels read: parity a, filter kind, cutoff-class index. A hybrid
// field's class holds its exponential tables and alt_cls its Gaussian ones (alt_cls = cls for the
// other kinds).
struct VarInfo {
  int parity;
  int kind;
  int cls;
  int alt_cls;
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
  int async_ok;       // input 16-byte aligned: shells may be copied with cp.async
  int var_begin;      // fields [var_begin, var_begin + var_count) are filtered (pointers are to
  int var_count;      // the whole state)
  int hybrid;         // some field of the launch takes the hybrid filter (every row is loaded)
  const int* list;    // grid indices (i * var_count + v - var_begin) of the launch's shells, or null for all
  int nlist;          // entries of list
};

// Arguments of the staged shell kernel (shell_kernel.cuh). Tables hold FP64 values, or
// FP32 pairs (hi, lo) for the compensated FP32 precision.
struct ShellArgs2 {
  int Nr, Nth, Nph, nvars;
  int ldS;                    // row stride of the staged shell (elements)
  int batch_th, batch_ph;     // sequences per FFT batch (sizes the scratch buffer)
  Factors f_th, f_ph;         // radices (2, 3, 4, 8) of 2 Ntheta and Nphi
  Factors f_sp;               // radices of Ntheta (the spectral form's per-mode transforms)
  const double* lmax;         // [ncls][Nr]
  const VarInfo* var;         // [nvars]
  const uint8_t* ring_info;   // [ncls][Nr][Nth]: bit 0 ring active, bit 1 mirror ring differs
  const void* g_th;           // [ncls][Nr][Nth+1]       f(l, l_max) / (2 Ntheta)
  const void* g_ph;           // [ncls][Nr][Nth][Nph/2+1] f(m, m_max) / Nphi
  const void* tw_th;          // [2 Nth] exp(-2 pi i n / (2 Nth))
  const void* tw_ph;          // [Nph]   exp(-2 pi i n / Nph)
  const void* consts;         // [2] sqrt(1/2), sqrt(3)/2
  unsigned* status;
  double eps;                 // epsilon of Jameson's detector (hybrid fields)
  float eps_m;                // eps = eps_m 2^eps_p, eps_m an FP32 rounding of its significand (the
  int eps_p;                  // detector's FP32 screen scales it without FP64 arithmetic)
};

// Instantiations of the staged shell kernel, one per (compensated precision?, FFT length, hybrid
// variant); defined by shell_inst.cu compiled once per triple. The single-CTA kernel's hybrid
// variant (HYB = 1) exists for the lengths a single CTA holds (not 256).
template <int DFP, int LEN, int HYB>
cudaError_t launch_shell_inst(const ShellArgs2& a, int threads, size_t smem, const LaunchIO& io, cudaStream_t s);
template <int DFP, int LEN, int HYB>
cudaError_t set_attr_inst(int bytes);
#define SPH_DECLARE_SHELL_INST(D, L, H)                                                                    \
  template <>                                                                                              \
  cudaError_t launch_shell_inst<D, L, H>(const ShellArgs2&, int, size_t, const LaunchIO&, cudaStream_t); \
  template <>                                                                                              \
  cudaError_t set_attr_inst<D, L, H>(int);
#define SPH_DECLARE_SHELL_INST_2(D, L) SPH_DECLARE_SHELL_INST(D, L, 0) SPH_DECLARE_SHELL_INST(D, L, 1)
SPH_DECLARE_SHELL_INST_2(0, 0)
SPH_DECLARE_SHELL_INST_2(0, 32)
SPH_DECLARE_SHELL_INST_2(0, 64)
SPH_DECLARE_SHELL_INST_2(0, 96)
SPH_DECLARE_SHELL_INST_2(0, 128)
SPH_DECLARE_SHELL_INST_2(0, 192)
SPH_DECLARE_SHELL_INST(0, 256, 0)
SPH_DECLARE_SHELL_INST_2(1, 0)
SPH_DECLARE_SHELL_INST_2(1, 32)
SPH_DECLARE_SHELL_INST_2(1, 64)
SPH_DECLARE_SHELL_INST_2(1, 96)
SPH_DECLARE_SHELL_INST_2(1, 128)
SPH_DECLARE_SHELL_INST_2(1, 192)
SPH_DECLARE_SHELL_INST(1, 256, 0)
SPH_DECLARE_SHELL_INST(2, 0, 0)    // FP64 spectral form (generic lengths)
SPH_DECLARE_SHELL_INST(2, 128, 0)  // FP64 spectral form, 2 Ntheta = Nphi = 128
#undef SPH_DECLARE_SHELL_INST_2
#undef SPH_DECLARE_SHELL_INST
// Cluster-pair instantiations for shells too large for one CTA (lengths 256 and generic), with and
// without the hybrid variant.
template <int DFP, int LEN, int HYB>
cudaError_t launch_shell_cl_inst(const ShellArgs2& a, int threads, size_t smem, const LaunchIO& io, cudaStream_t s);
template <int DFP, int LEN, int HYB>
cudaError_t set_attr_cl_inst(int bytes);
#define SPH_DECLARE_SHELL_CL_INST(D, L, H)                                                                    \
  template <>                                                                                                 \
  cudaError_t launch_shell_cl_inst<D, L, H>(const ShellArgs2&, int, size_t, const LaunchIO&, cudaStream_t); \
  template <>                                                                                                 \
  cudaError_t set_attr_cl_inst<D, L, H>(int);
SPH_DECLARE_SHELL_CL_INST(0, 0, 0)
SPH_DECLARE_SHELL_CL_INST(0, 0, 1)
SPH_DECLARE_SHELL_CL_INST(0, 256, 0)
SPH_DECLARE_SHELL_CL_INST(0, 256, 1)
SPH_DECLARE_SHELL_CL_INST(1, 0, 0)
SPH_DECLARE_SHELL_CL_INST(1, 0, 1)
SPH_DECLARE_SHELL_CL_INST(1, 256, 0)
SPH_DECLARE_SHELL_CL_INST(1, 256, 1)
#undef SPH_DECLARE_SHELL_CL_INST
size_t shell_smem_cl_bytes(const ShellArgs2& a, int precision);
cudaError_t launch_shell_cl(const ShellArgs2& a, int precision, int threads, size_t smem, const LaunchIO& io,
                            cudaStream_t s);

// Units kernel (ring pairs of sparse shells, single-CTA plans): per (precision, length) in the
// non-hybrid instantiation objects; the shell copy for out-of-place calls.
template <int DFP, int LEN>
cudaError_t launch_units_inst(const ShellArgs2& a, size_t smem, const LaunchIO& io, const int* units, int nunits,
                              cudaStream_t s);
template <int DFP, int LEN>
cudaError_t set_attr_units_inst(int bytes);
#define SPH_DECLARE_UNITS_INST(D, L)                                                                              \
  template <>                                                                                                     \
  cudaError_t launch_units_inst<D, L>(const ShellArgs2&, size_t, const LaunchIO&, const int*, int, cudaStream_t); \
  template <>                                                                                                     \
  cudaError_t set_attr_units_inst<D, L>(int);
SPH_DECLARE_UNITS_INST(0, 0)
SPH_DECLARE_UNITS_INST(0, 32)
SPH_DECLARE_UNITS_INST(0, 64)
SPH_DECLARE_UNITS_INST(0, 96)
SPH_DECLARE_UNITS_INST(0, 128)
SPH_DECLARE_UNITS_INST(0, 192)
SPH_DECLARE_UNITS_INST(1, 0)
SPH_DECLARE_UNITS_INST(1, 32)
SPH_DECLARE_UNITS_INST(1, 64)
SPH_DECLARE_UNITS_INST(1, 96)
SPH_DECLARE_UNITS_INST(1, 128)
SPH_DECLARE_UNITS_INST(1, 192)
#undef SPH_DECLARE_UNITS_INST
size_t units_smem_bytes(const ShellArgs2& a, int precision);
cudaError_t launch_units(const ShellArgs2& a, int precision, size_t smem, const LaunchIO& io, const int* units,
                         int nunits, cudaStream_t s);
cudaError_t launch_copy_shells(const double* in, double* out, const int* list, int nshells, size_t shell_values,
                               cudaStream_t s);

size_t shell_smem_bytes(const ShellArgs2& a, int precision);
int fixed_length(const ShellArgs2& a);
Factors kernel_radices(const ShellArgs2& a, int N, int precision);
cudaError_t launch_shell(const ShellArgs2& a, int precision, int threads, size_t smem, const LaunchIO& io,
                         cudaStream_t s);
cudaError_t set_shell_smem_attr(int device);

}  // namespace sph

namespace sph {
struct TcPlan;
}

struct sph_filter_plan_s {
  int device = 0;
  int Nr = 0, Nth = 0, Nph = 0, nvars = 0, precision = 0;
  double dr_min = 1.0, floor_ = 2.0;
  std::vector<int> parity, kind, var_cls;
  std::vector<double> L, r;
  int ncls = 0;
  bool has_hybrid = false;
  std::vector<int> cls_kind;
  std::vector<double> cls_L;
  std::vector<double> h_lmax, h_mmax;

  sph::ShellArgs args{};
  size_t smem_bytes = 0;
  int launches = 1;
  std::atomic<long long> launched{0};  // kernel launches enqueued so far (captures count once)

  // staged shell kernel (used when the shape fits it)
  bool use_v2 = false;
  bool cluster = false;       // a 2-CTA cluster filters each shell
  // Split launch (single-CTA plans): shells whose theta pass is the identity ("sparse") are copied
  // in -> out and only their active ring pairs are filtered, by the units kernel, several shells'
  // pairs per CTA; the other ("dense") shells run the shell kernel from a list. Per field v, its
  // entries are [off[v], off[v + 1]) of each list.
  // The copy and the units kernel run on side streams of the plan, beside the shell kernel on
  // the caller's stream: forked from it and joined back by events (split_mu orders the calls that
  // share them). The copy, bound by memory, runs on a high-priority stream so that it overlaps the
  // shell kernel's arithmetic early; the units kernel follows it on a normal-priority stream.
  bool split = false;
  cudaStream_t side = nullptr, side_copy = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_copy = nullptr, ev_join = nullptr;
  std::mutex split_mu;
  int* d_dense = nullptr;     // i * nvars + v (the shell kernel's grid index over all fields)
  int* d_sparse = nullptr;    // v * Nr + i
  int* d_units = nullptr;     // (v * Nr + i) * Ntheta + j: ring pair (j, Ntheta - 1 - j), one active
  std::vector<int> dense_off, sparse_off, units_off;
  size_t smem_units = 0;
  sph::ShellArgs2 args2{};
  int threads2 = 0;
  size_t smem2 = 0;
  void* d_tabs = nullptr;     // one allocation holding every v2 table

  double* d_lmax = nullptr;
  double* d_mmax = nullptr;
  sph::VarInfo* d_var = nullptr;
  double2* d_tw_th = nullptr;
  double2* d_tw_ph = nullptr;
  unsigned* d_status = nullptr;

  // split-precision tensor-core form (SPH_PREC_SPLIT_TC)
  sph::TcPlan* tc = nullptr;

  // staging buffers and pipeline streams of sph_filter_apply_host (created on first use)
  double* d_stage_in = nullptr;
  double* d_stage_out = nullptr;
  // host-buffer pipeline: one stream for the copies in, one for the copies out, kPipeStreams compute
  // streams (the tensor-core form uses the first three, one per counter set); the call's start and
  // end events, and per chunk (at most one per field) an event after its copy in and one after its
  // kernels
  static constexpr int kPipeStreams = 6;
  cudaStream_t pipe[kPipeStreams] = {};
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_start = nullptr, pipe_end = nullptr;
  std::vector<cudaEvent_t> chunk_in, chunk_done;
};

namespace sph {
// Filter function f(|l|, l_max) of Sec. II.C in extended precision.
long double filter_value(int kind, long double al, long double lmax);

// Split-precision tensor-core form (tc.cu): tables at plan creation, release, and one application
// (theta then phi pass, or the reverse for the transpose) of the fields [var_begin, var_begin +
// var_count) from in to out (in == out allowed). The form keeps no state between launches (its
// working set lives in each CTA's shared and tensor memory), so calls may overlap on any streams;
// `set` is unused. *nlaunch (if not null) receives the number of kernels enqueued.
sph_status tc_setup(sph_filter_plan_s* p);
void tc_free(sph_filter_plan_s* p);
sph_status tc_reserve_pipeline(sph_filter_plan_s* p);
cudaError_t tc_launch(sph_filter_plan_s* p, const double* in, double* out, int transpose, int var_begin,
                      int var_count, cudaStream_t s, int set, int* nlaunch = nullptr);

// Several tensor-core plans filtered by one persistent launch per application (tc.cu): a merged work
// list over the grids and one set of counters (launches of one batch must not overlap).
struct TcBatch;
sph_status tc_batch_setup(TcBatch** out, sph_filter_plan_s* const* plans, int nplans);
void tc_batch_free(TcBatch* b);
cudaError_t tc_batch_launch(TcBatch* b, const double* const* in, double* const* out, cudaStream_t s);

// Enqueue one filter application of a plan (validates pointers; see sph_filter_apply).
sph_status launch_plan(sph_filter_plan_s* p, const void* in, const void* aux, void* out, int map_in, int map_out,
                       int transpose, int is_f32, cudaStream_t stream);
// The same for the fields [var_begin, var_begin + var_count) only. tc_set: the tensor-core form's
// scratch set (0 for every caller but the host-buffer pipeline, which passes 1..3 by stream).
sph_status launch_plan_vars(sph_filter_plan_s* p, const void* in, const void* aux, void* out, int map_in,
                            int map_out, int transpose, int is_f32, int var_begin, int var_count,
                            cudaStream_t stream, int tc_set = 0);
// Shared-memory bytes the plain shell kernel needs for this plan's shape (0 if it cannot fit).
size_t plain_smem_bytes(const ShellArgs& a, int* chunk_th, int* chunk_ph);
// Enqueue the plain FP64 shell kernel.
cudaError_t launch_plain(const sph_filter_plan_s& p, const LaunchIO& io, cudaStream_t s);
// Largest dynamic shared memory a CTA may use on this device.
int max_smem_optin(int device);
}  // namespace sph
