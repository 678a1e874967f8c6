// Selection among the compiled instantiations of the staged shell kernel.
#include "shell_kernel.cuh"

namespace sph {

int fixed_length(const ShellArgs2& a) {
  const int L = a.Nph;
  if (2 * a.Nth != L) return 0;
  if (L == 32 || L == 64 || L == 96 || L == 128 || L == 192 || L == 256) return L;
  return 0;
}

size_t shell_smem_bytes(const ShellArgs2& a, int precision) {
  return precision == SPH_PREC_F32X2 ? shellk::smem_impl<shellk::DF>(a) : shellk::smem_impl<shellk::F64>(a);
}

template <int DFP, int HYB>
static cudaError_t launch_p(const ShellArgs2& a, int threads, size_t smem, const LaunchIO& io, cudaStream_t s) {
  switch (fixed_length(a)) {
    case 32: return launch_shell_inst<DFP, 32, HYB>(a, threads, smem, io, s);
    case 64: return launch_shell_inst<DFP, 64, HYB>(a, threads, smem, io, s);
    case 96: return launch_shell_inst<DFP, 96, HYB>(a, threads, smem, io, s);
    case 128: return launch_shell_inst<DFP, 128, HYB>(a, threads, smem, io, s);
    case 192: return launch_shell_inst<DFP, 192, HYB>(a, threads, smem, io, s);
    case 256:  // 128 x 256 shells run on CTA pairs, which take no hybrid fields
      if (HYB) return cudaErrorInvalidValue;
      return launch_shell_inst<DFP, 256, 0>(a, threads, smem, io, s);
    default: return launch_shell_inst<DFP, 0, HYB>(a, threads, smem, io, s);
  }
}

cudaError_t launch_shell(const ShellArgs2& a, int precision, int threads, size_t smem, const LaunchIO& io,
                         cudaStream_t s) {
  // launches with hybrid fields run the kernel variant that has their detector and tables
  if (precision == SPH_PREC_F32X2)
    return io.hybrid ? launch_p<1, 1>(a, threads, smem, io, s) : launch_p<1, 0>(a, threads, smem, io, s);
  return io.hybrid ? launch_p<0, 1>(a, threads, smem, io, s) : launch_p<0, 0>(a, threads, smem, io, s);
}

size_t shell_smem_cl_bytes(const ShellArgs2& a, int precision) {
  return precision == SPH_PREC_F32X2 ? shellk::shell_smem_cl<shellk::DF>(a) : shellk::shell_smem_cl<shellk::F64>(a);
}

cudaError_t launch_shell_cl(const ShellArgs2& a, int precision, int threads, size_t smem, const LaunchIO& io,
                            cudaStream_t s) {
  const bool fixed = fixed_length(a) == 256;
  if (precision == SPH_PREC_F32X2) {
    if (io.hybrid)
      return fixed ? launch_shell_cl_inst<1, 256, 1>(a, threads, smem, io, s) : launch_shell_cl_inst<1, 0, 1>(a, threads, smem, io, s);
    return fixed ? launch_shell_cl_inst<1, 256, 0>(a, threads, smem, io, s) : launch_shell_cl_inst<1, 0, 0>(a, threads, smem, io, s);
  }
  if (io.hybrid)
    return fixed ? launch_shell_cl_inst<0, 256, 1>(a, threads, smem, io, s) : launch_shell_cl_inst<0, 0, 1>(a, threads, smem, io, s);
  return fixed ? launch_shell_cl_inst<0, 256, 0>(a, threads, smem, io, s) : launch_shell_cl_inst<0, 0, 0>(a, threads, smem, io, s);
}

template <int DFP>
static cudaError_t set_attr_p(int bytes) {
  cudaError_t e = cudaSuccess;
  auto both = [&](cudaError_t (*f0)(int), cudaError_t (*f1)(int)) {
    if (e == cudaSuccess) e = f0(bytes);
    if (e == cudaSuccess && f1) e = f1(bytes);
  };
  both(set_attr_inst<DFP, 0, 0>, set_attr_inst<DFP, 0, 1>);
  both(set_attr_inst<DFP, 32, 0>, set_attr_inst<DFP, 32, 1>);
  both(set_attr_inst<DFP, 64, 0>, set_attr_inst<DFP, 64, 1>);
  both(set_attr_inst<DFP, 96, 0>, set_attr_inst<DFP, 96, 1>);
  both(set_attr_inst<DFP, 128, 0>, set_attr_inst<DFP, 128, 1>);
  both(set_attr_inst<DFP, 192, 0>, set_attr_inst<DFP, 192, 1>);
  both(set_attr_inst<DFP, 256, 0>, nullptr);
  both(set_attr_cl_inst<DFP, 0, 0>, set_attr_cl_inst<DFP, 0, 1>);
  both(set_attr_cl_inst<DFP, 256, 0>, set_attr_cl_inst<DFP, 256, 1>);
  return e;
}

cudaError_t set_shell_smem_attr(int device) {
  const int bytes = max_smem_optin(device);
  cudaError_t e = set_attr_p<0>(bytes);
  if (e != cudaSuccess) return e;
  return set_attr_p<1>(bytes);
}

}  // namespace sph
