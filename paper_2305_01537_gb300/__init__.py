"""GB300-native double FFT filter (arXiv:2305.01537, Sec. II.C) for fields on spherical grids.

The compute path is the CUDA library libsph_filter.so behind the C ABI of include/sph_filter.h;
`binding` marshals arguments to it. PyTorch provides device memory and streams only.
"""
from .binding import (Plan, Batch, SphFilterError, SPH_FILTER_EXP, SPH_FILTER_GAUSS, SPH_FILTER_SHARP, SPH_FILTER_HYBRID,
                      SPH_PREC_F64, SPH_PREC_SPLIT_TC, SPH_PREC_F32X2, SPH_PREC_SPECTRAL, load, enforce_constraints)

__all__ = ["Plan", "Batch", "SphFilterError", "SPH_FILTER_EXP", "SPH_FILTER_GAUSS", "SPH_FILTER_SHARP", "SPH_FILTER_HYBRID",
           "SPH_PREC_F64", "SPH_PREC_SPLIT_TC", "SPH_PREC_F32X2", "SPH_PREC_SPECTRAL", "load", "enforce_constraints"]
