// Host-buffer filter call that allocates no device memory: the device staging of
// sph_filter_apply_host lives in a fixed array of this file instead of buffers the plan allocates.
//
// Why: some callers cannot let a library call cudaMalloc. A simulation framework that reserves the
// whole device memory for its own allocator at start-up leaves nothing for the library to allocate
// (and a late allocation would fail or fragment its pool); code that must not synchronise the
// device at that point cannot afford cudaMalloc/cudaFree either, since they may synchronise.
//
// The array is a file-scope __device__ variable of 32 MiB. With lazy module loading (the CUDA
// default), a device gets that memory when this file's module is first loaded there, which is the
// first call of this entry point on that device (the first cudaGetSymbolAddress below); it is then
// held until the process exits. Host code cannot use the variable's name as a device address; the
// address is looked up with cudaGetSymbolAddress, on every call (cheap once the module is loaded), so
// that a cudaDeviceReset between calls cannot leave a stale address behind.
#include <cstdint>

#include "internal.h"

namespace {

// Largest state the call accepts, in points; the array holds the input and the output.
constexpr long long kNoAllocMaxPoints = 1LL << 21;  // 2,097,152 points = 16 MiB per direction

static __device__ __align__(256) double g_noalloc_stage[2 * kNoAllocMaxPoints];

// Device address of the staging array on the current device.
sph_status stage_address(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_stage) != cudaSuccess || !p) return SPH_ECUDA;
  *out = static_cast<double*>(p);
  return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_filter_apply_host_noalloc(sph_filter_plan plan, const double* host_in, double* host_out,
                                                    sph_stream_t stream) {
  if (!plan || !host_in || !host_out) return SPH_EINVAL;
  const long long n = sph_filter_plan_points(plan);
  if (n > kNoAllocMaxPoints) return SPH_EINVAL;  // larger than the fixed staging array
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return SPH_ECUDA;
  if (cur != plan->device && cudaSetDevice(plan->device) != cudaSuccess) return SPH_ECUDA;
  double* stage = nullptr;
  sph_status st = stage_address(&stage);
  if (st == SPH_OK) {
    double* d_in = stage;
    double* d_out = stage + kNoAllocMaxPoints;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(d_in, host_in, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess)
      st = SPH_ECUDA;
    if (st == SPH_OK) st = sph::launch_plan(plan, d_in, nullptr, d_out, sph::kMapNone, sph::kOutNone, 0, 0, s);
    if (st == SPH_OK &&
        cudaMemcpyAsync(host_out, d_out, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = SPH_ECUDA;
  }
  if (cur != plan->device) cudaSetDevice(cur);
  return st;
}
