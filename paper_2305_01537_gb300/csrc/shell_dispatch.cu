// Selection among the compiled instantiations of the staged shell kernel.
#include "shell_kernel.cuh"

namespace sph {

int fixed_length(const ShellArgs2& a) {
  const int L = a.Nph;
  if (2 * a.Nth != L) return 0;
  if (L == 32 || L == 64 || L == 96 || L == 128 || L == 192 || L == 256) return L;
  return 0;
}

// The radix sequence the compiled kernels run for a transform of length N (2 Ntheta or Nphi): the
// compiled sequence of run_pass for the fixed lengths, else the plan's factorisation. The twiddle
// tables are laid out stage by stage in this order.
Factors kernel_radices(const ShellArgs2& a, int N, int precision) {
  Factors f = N == 2 * a.Nth ? a.f_th : a.f_ph;
  const int L = fixed_length(a);
  if (L != 0) {
    static const int r32[] = {8, 4}, r64[] = {8, 8}, r96[] = {8, 4, 3}, r128d[] = {8, 4, 4}, r128[] = {8, 8, 2},
                     r192[] = {8, 8, 3}, r256[] = {8, 8, 4};
    const int* r = L == 32 ? r32 : L == 64 ? r64 : L == 96 ? r96 : L == 192 ? r192 : L == 256 ? r256
                 : (precision == SPH_PREC_F32X2 ? r128d : r128);
    f.n = L;
    f.nst = L == 32 || L == 64 ? 2 : 3;
    for (int s = 0; s < f.nst; ++s) f.radix[s] = r[s];
  }
  return f;
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
  if (precision == SPH_PREC_SPECTRAL) {
    // the FP64 spectral form (plans with hybrid fields are rejected at creation)
    if (io.hybrid) return cudaErrorInvalidValue;
    return fixed_length(a) == 128 ? launch_shell_inst<2, 128, 0>(a, threads, smem, io, s)
                                  : launch_shell_inst<2, 0, 0>(a, threads, smem, io, s);
  }
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

size_t units_smem_bytes(const ShellArgs2& a, int) { return shellk::units_smem(a); }

template <int DFP>
static cudaError_t launch_units_p(const ShellArgs2& a, size_t smem, const LaunchIO& io, const int* units, int n,
                                  cudaStream_t s) {
  switch (fixed_length(a)) {
    case 32: return launch_units_inst<DFP, 32>(a, smem, io, units, n, s);
    case 64: return launch_units_inst<DFP, 64>(a, smem, io, units, n, s);
    case 96: return launch_units_inst<DFP, 96>(a, smem, io, units, n, s);
    case 128: return launch_units_inst<DFP, 128>(a, smem, io, units, n, s);
    case 192: return launch_units_inst<DFP, 192>(a, smem, io, units, n, s);
    case 256: return cudaErrorInvalidValue;  // 128 x 256 shells run on CTA pairs, without units
    default: return launch_units_inst<DFP, 0>(a, smem, io, units, n, s);
  }
}

cudaError_t launch_units(const ShellArgs2& a, int precision, size_t smem, const LaunchIO& io, const int* units,
                         int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  return precision == SPH_PREC_F32X2 ? launch_units_p<1>(a, smem, io, units, nunits, s)
                                     : launch_units_p<0>(a, smem, io, units, nunits, s);
}

// Copies whole shells in -> out (the sparse shells of an out-of-place call; the units kernel then
// overwrites their active rows): one CTA per listed shell, 16-byte pieces.
__global__ void __launch_bounds__(256) copy_shells_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                                          const int* list, int shell_pairs) {
  const size_t base = (size_t)list[blockIdx.x] * (size_t)shell_pairs;
  for (int c = threadIdx.x; c < shell_pairs; c += blockDim.x) __stcs(out + base + c, __ldcs(in + base + c));
}

cudaError_t launch_copy_shells(const double* in, double* out, const int* list, int nshells, size_t shell_values,
                               cudaStream_t s) {
  if (nshells <= 0) return cudaSuccess;
  copy_shells_kernel<<<(unsigned)nshells, 256, 0, s>>>(reinterpret_cast<const double2*>(in),
                                                       reinterpret_cast<double2*>(out), list, (int)(shell_values / 2));
  return cudaGetLastError();
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
  both(set_attr_units_inst<DFP, 0>, set_attr_units_inst<DFP, 32>);
  both(set_attr_units_inst<DFP, 64>, set_attr_units_inst<DFP, 96>);
  both(set_attr_units_inst<DFP, 128>, set_attr_units_inst<DFP, 192>);
  both(set_attr_cl_inst<DFP, 0, 0>, set_attr_cl_inst<DFP, 0, 1>);
  both(set_attr_cl_inst<DFP, 256, 0>, set_attr_cl_inst<DFP, 256, 1>);
  return e;
}

cudaError_t set_shell_smem_attr(int device) {
  const int bytes = max_smem_optin(device);
  cudaError_t e = set_attr_p<0>(bytes);
  if (e == cudaSuccess) e = set_attr_p<1>(bytes);
  if (e == cudaSuccess) e = set_attr_inst<2, 0, 0>(bytes);
  if (e == cudaSuccess) e = set_attr_inst<2, 128, 0>(bytes);
  return e;
}

}  // namespace sph
