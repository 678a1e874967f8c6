// One instantiation of the staged shell kernel. The build compiles this file once per
// (precision, FFT length, hybrid variant) triple with -DSPH_SHELL_DF=0|1|2
// -DSPH_SHELL_LEN=0|32|64|96|128|192|256 -DSPH_SHELL_HYB=0|1, so the instantiations compile in
// parallel; shell_dispatch.cu selects one at launch time. The cluster-pair kernel is instantiated
// for the lengths 256 and generic, in both variants; the spectral form (SPH_SHELL_DF=2) for the
// length 128 and generic lengths, single-CTA shells only.
#include "shell_kernel.cuh"

#ifndef SPH_SHELL_DF
#define SPH_SHELL_DF 0
#endif
#ifndef SPH_SHELL_LEN
#define SPH_SHELL_LEN 0
#endif
#ifndef SPH_SHELL_HYB
#define SPH_SHELL_HYB 0
#endif

namespace sph {

// SPH_SHELL_DF: 0 FP64, 1 compensated FP32 pairs, 2 the FP64 spectral form (shell kernel only)
#if SPH_SHELL_DF == 1
using InstPolicy = shellk::DF;
#else
using InstPolicy = shellk::F64;
#endif
constexpr bool kInstSpec = SPH_SHELL_DF == 2;

#if !(SPH_SHELL_HYB && SPH_SHELL_LEN == 256)  // 128 x 256 shells run on CTA pairs
template <>
cudaError_t launch_shell_inst<SPH_SHELL_DF, SPH_SHELL_LEN, SPH_SHELL_HYB>(const ShellArgs2& a, int threads, size_t smem,
                                                                        const LaunchIO& io, cudaStream_t s) {
  return shellk::launch_impl<InstPolicy, SPH_SHELL_LEN, SPH_SHELL_HYB != 0, kInstSpec>(a, threads, smem, io, s);
}

template <>
cudaError_t set_attr_inst<SPH_SHELL_DF, SPH_SHELL_LEN, SPH_SHELL_HYB>(int bytes) {
  return shellk::set_attr_impl<InstPolicy, SPH_SHELL_LEN, SPH_SHELL_HYB != 0, kInstSpec>(bytes);
}
#endif

#if SPH_SHELL_HYB == 0 && SPH_SHELL_LEN != 256 && SPH_SHELL_DF != 2
template <>
cudaError_t launch_units_inst<SPH_SHELL_DF, SPH_SHELL_LEN>(const ShellArgs2& a, size_t smem, const LaunchIO& io,
                                                         const int* units, int nunits, cudaStream_t s) {
  return shellk::launch_units_impl<InstPolicy, SPH_SHELL_LEN>(a, smem, io, units, nunits, s);
}

template <>
cudaError_t set_attr_units_inst<SPH_SHELL_DF, SPH_SHELL_LEN>(int bytes) {
  return shellk::set_attr_units_impl<InstPolicy, SPH_SHELL_LEN>(bytes);
}
#endif

#if (SPH_SHELL_LEN == 0 || SPH_SHELL_LEN == 256) && SPH_SHELL_DF != 2
template <>
cudaError_t launch_shell_cl_inst<SPH_SHELL_DF, SPH_SHELL_LEN, SPH_SHELL_HYB>(const ShellArgs2& a, int threads,
                                                                           size_t smem, const LaunchIO& io,
                                                                           cudaStream_t s) {
  return shellk::launch_cl_impl<InstPolicy, SPH_SHELL_LEN, SPH_SHELL_HYB != 0>(a, threads, smem, io, s);
}

template <>
cudaError_t set_attr_cl_inst<SPH_SHELL_DF, SPH_SHELL_LEN, SPH_SHELL_HYB>(int bytes) {
  return shellk::set_attr_cl_impl<InstPolicy, SPH_SHELL_LEN, SPH_SHELL_HYB != 0>(bytes);
}
#endif

}  // namespace sph
