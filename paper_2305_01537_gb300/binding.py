"""Thin Python binding of the sph_filter C ABI (include/sph_filter.h).

Only argument marshalling lives here: every step of the filter runs in the CUDA library. The
library must have been built (``python -m paper_2305_01537_gb300.build``); importing this module
without it raises, so nothing silently falls back to another implementation. PyTorch is used for
device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph_filter.so")

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_EUNSUPPORTED, SPH_ETIMEOUT, SPH_EALIAS, SPH_EDEVICE = range(8)
SPH_FILTER_EXP, SPH_FILTER_GAUSS, SPH_FILTER_SHARP, SPH_FILTER_HYBRID = 0, 1, 2, 3
SPH_PREC_F64, SPH_PREC_SPLIT_TC, SPH_PREC_F32X2, SPH_PREC_SPECTRAL = 0, 1, 2, 3

# Every symbol include/sph_filter.h declares (checked by the tests).
EXPORTED = (
    "sph_filter_plan_create", "sph_filter_plan_destroy", "sph_filter_apply", "sph_filter_apply_adjoint",
    "sph_filter_apply_tanh", "sph_filter_apply_adjoint_tanh", "sph_filter_apply_f32",
    "sph_filter_apply_adjoint_f32", "sph_filter_apply_tanh_f32", "sph_filter_apply_adjoint_tanh_f32",
    "sph_filter_apply_host", "sph_filter_plan_sync_status", "sph_filter_plan_points",
    "sph_filter_plan_launches", "sph_filter_status_string", "sph_filter_batch_create",
    "sph_filter_batch_destroy", "sph_filter_batch_apply", "sph_filter_batch_capture", "sph_filter_batch_launch",
    "sph_filter_plan_autotune", "sph_filter_apply_host_noalloc", "sph_filter_plan_launch_count",
    "sph_enforce_constraints",
)


class SphFilterError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {sph_filter_status_string(status)} (status {status})")


class sph_cutoff_params(ctypes.Structure):
    _fields_ = [("r", ctypes.c_void_p), ("dr_min", ctypes.c_double), ("L", ctypes.c_void_p),
                ("kind", ctypes.c_void_p), ("floor", ctypes.c_double), ("precision", ctypes.c_int),
                ("eps", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Load the built library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2305_01537_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    sig = {
        "sph_filter_plan_create": ([ctypes.POINTER(P), I, I, I, I, P, ctypes.POINTER(sph_cutoff_params)], I),
        "sph_filter_plan_destroy": ([P], None),
        "sph_filter_apply": ([P, P, P, P], I),
        "sph_filter_apply_adjoint": ([P, P, P, P], I),
        "sph_filter_apply_tanh": ([P, P, P, P], I),
        "sph_filter_apply_adjoint_tanh": ([P, P, P, P, P], I),
        "sph_filter_apply_f32": ([P, P, P, P], I),
        "sph_filter_apply_adjoint_f32": ([P, P, P, P], I),
        "sph_filter_apply_tanh_f32": ([P, P, P, P], I),
        "sph_filter_apply_adjoint_tanh_f32": ([P, P, P, P, P], I),
        "sph_filter_apply_host": ([P, P, P, P], I),
        "sph_filter_plan_sync_status": ([P], I),
        "sph_filter_plan_points": ([P], LL),
        "sph_filter_plan_launches": ([P], I),
        "sph_filter_plan_launch_count": ([P], LL),
        "sph_enforce_constraints": ([P, I, I, I, I, P, P, I, P, ctypes.c_double, P], I),
        "sph_filter_status_string": ([I], ctypes.c_char_p),
        "sph_filter_batch_create": ([ctypes.POINTER(P), I, P], I),
        "sph_filter_batch_destroy": ([P], None),
        "sph_filter_batch_apply": ([P, P, P, P], I),
        "sph_filter_batch_capture": ([P, P, P, I, P], I),
        "sph_filter_batch_launch": ([P, P], I),
        "sph_filter_plan_autotune": ([P, P, P, P, ctypes.POINTER(ctypes.c_double)], I),
        "sph_filter_apply_host_noalloc": ([P, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def sph_filter_status_string(status: int) -> str:
    return load().sph_filter_status_string(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != SPH_OK:
        raise SphFilterError(status, where)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A filter plan (sph_filter_plan_create) for states of shape [nvars, Nr, Ntheta, Nphi]."""

    def __init__(self, Nr: int, Ntheta: int, Nphi: int, parity: Sequence[int], kind: Sequence[int],
                 L: Sequence[float], r: Sequence[float], dr_min: float = 1.0, floor: float = 2.0,
                 precision: int = SPH_PREC_F64, eps: float = 1e-12):
        """eps: epsilon of Jameson's detector for SPH_FILTER_HYBRID fields."""
        lib = load()
        self.Nr, self.Ntheta, self.Nphi = int(Nr), int(Ntheta), int(Nphi)
        self.nvars = len(parity)
        self._parity = np.ascontiguousarray(parity, dtype=np.int32)
        self._kind = np.ascontiguousarray(kind, dtype=np.int32)
        self._L = np.ascontiguousarray(L, dtype=np.float64)
        self._r = np.ascontiguousarray(r, dtype=np.float64)
        if self._kind.shape != (self.nvars,) or self._L.shape != (self.nvars,) or self._r.shape != (self.Nr,):
            raise ValueError("kind and L need nvars entries, r needs Nr entries")
        prm = sph_cutoff_params(self._r.ctypes.data, float(dr_min), self._L.ctypes.data, self._kind.ctypes.data,
                                float(floor), int(precision), float(eps))
        h = ctypes.c_void_p()
        _check(lib.sph_filter_plan_create(ctypes.byref(h), self.Nr, self.Ntheta, self.Nphi, self.nvars,
                                          self._parity.ctypes.data, ctypes.byref(prm)), "sph_filter_plan_create")
        self._h = h
        import torch
        self.device = torch.cuda.current_device()  # the device sph_filter_plan_create bound the plan to
        self.precision = int(precision)

    @classmethod
    def from_grid(cls, grid, precision: int = SPH_PREC_F64) -> "Plan":
        return cls(grid.Nr, grid.Ntheta, grid.Nphi, grid.parity, grid.kind, grid.L, grid.r, grid.dr_min,
                   grid.floor, precision, getattr(grid, "eps", 1e-12))

    @property
    def shape(self):
        return (self.nvars, self.Nr, self.Ntheta, self.Nphi)

    @property
    def points(self) -> int:
        return int(load().sph_filter_plan_points(self._h))

    @property
    def launches(self) -> int:
        return int(load().sph_filter_plan_launches(self._h))

    @property
    def launch_count(self) -> int:
        """Kernel launches this plan has enqueued so far (graph captures count once)."""
        return int(load().sph_filter_plan_launch_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().sph_filter_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- device-resident calls -------------------------------------------------------------
    def _io(self, x, out, dtype):
        import torch
        if not (x.is_cuda and x.dtype == dtype and x.is_contiguous() and tuple(x.shape) == self.shape):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of shape {self.shape}")
        if x.device.index != self.device:
            raise ValueError(f"the tensor is on cuda:{x.device.index}, the plan on cuda:{self.device}")
        if out is None:
            with torch.cuda.device(self.device):
                out = torch.empty_like(x)
        elif not (out.is_cuda and out.dtype == dtype and out.is_contiguous() and tuple(out.shape) == self.shape
                  and out.device.index == self.device):
            raise ValueError("out must match the input (shape, dtype, layout and device)")
        return out

    def _call(self, fname, x, out, stream, aux=None):
        import torch
        dtype = torch.float32 if fname.endswith("_f32") else torch.float64
        out = self._io(x, out, dtype)
        fn = getattr(load(), fname)
        with torch.cuda.device(self.device):
            if aux is None:
                st = fn(self._h, x.data_ptr(), out.data_ptr(), _stream_handle(stream))
            else:
                self._io(aux, aux, dtype)
                st = fn(self._h, x.data_ptr(), aux.data_ptr(), out.data_ptr(), _stream_handle(stream))
        _check(st, fname)
        return out

    def apply(self, x, out=None, stream=None):
        """out = F x (sph_filter_apply / sph_filter_apply_f32 by dtype)."""
        return self._call("sph_filter_apply" + ("_f32" if _is_f32(x) else ""), x, out, stream)

    def apply_adjoint(self, x, out=None, stream=None):
        """out = F^T x."""
        return self._call("sph_filter_apply_adjoint" + ("_f32" if _is_f32(x) else ""), x, out, stream)

    def apply_tanh(self, z, out=None, stream=None):
        """out = F(tanh(z))."""
        return self._call("sph_filter_apply_tanh" + ("_f32" if _is_f32(z) else ""), z, out, stream)

    def apply_adjoint_tanh(self, g, z, out=None, stream=None):
        """out = (1 - tanh(z)^2) * F^T g."""
        return self._call("sph_filter_apply_adjoint_tanh" + ("_f32" if _is_f32(g) else ""), g, out, stream, aux=z)

    # -- host-resident call ----------------------------------------------------------------
    def apply_host(self, x_host, out_host, stream=None):
        """sph_filter_apply_host: host (ideally pinned) FP64 tensors in and out; asynchronous."""
        import torch
        for t in (x_host, out_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != self.shape:
                raise ValueError(f"expected contiguous host float64 tensors of shape {self.shape}")
        _check(load().sph_filter_apply_host(self._h, x_host.data_ptr(), out_host.data_ptr(), _stream_handle(stream)),
               "sph_filter_apply_host")
        return out_host

    def sync_status(self) -> int:
        return int(load().sph_filter_plan_sync_status(self._h))

    def autotune(self, x, out, stream=None) -> float:
        """sph_filter_plan_autotune on the given FP64 device buffers; returns the best time (ms)."""
        import torch
        self._io(x, out, torch.float64)
        best = ctypes.c_double(0.0)
        _check(load().sph_filter_plan_autotune(self._h, x.data_ptr(), out.data_ptr(), _stream_handle(stream),
                                               ctypes.byref(best)), "sph_filter_plan_autotune")
        return best.value


class Batch:
    """sph_filter_batch: several plans (grids) filtered by one call, or replayed as a CUDA graph."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(load().sph_filter_batch_create(ctypes.byref(h), len(self.plans), arr), "sph_filter_batch_create")
        self._h = h

    def _ptrs(self, xs, outs):
        import torch
        if len(xs) != len(self.plans) or len(outs) != len(self.plans):
            raise ValueError("one input and one output per plan")
        for p, x, o in zip(self.plans, xs, outs):
            p._io(x, o, torch.float64)
        ins = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        ous = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        return ins, ous

    def apply(self, xs, outs, stream=None):
        ins, ous = self._ptrs(xs, outs)
        _check(load().sph_filter_batch_apply(self._h, ins, ous, _stream_handle(stream)), "sph_filter_batch_apply")
        return outs

    def capture(self, xs, outs, napply: int, stream=None):
        ins, ous = self._ptrs(xs, outs)
        self._keep = (xs, outs)
        _check(load().sph_filter_batch_capture(self._h, ins, ous, int(napply), _stream_handle(stream)),
               "sph_filter_batch_capture")

    def launch(self, stream=None):
        _check(load().sph_filter_batch_launch(self._h, _stream_handle(stream)), "sph_filter_batch_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().sph_filter_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _is_f32(t) -> bool:
    import torch
    return t.dtype == torch.float32


def enforce_constraints(state, h_vars: Sequence[int], a_vars: Sequence[int], alpha_var: int,
                        theta_filtered=None, alpha_bh: float = 0.3, stream=None):
    """sph_enforce_constraints, in place on a CUDA float64 state [nvars, Nr, Ntheta, Nphi].

    h_vars, a_vars: 6 field indices each (11, 12, 13, 22, 23, 33); theta_filtered: a CUDA uint8 (or
    bool) tensor of Nr flags, or None. Returns the state."""
    import torch
    if not state.is_cuda or state.dtype != torch.float64 or not state.is_contiguous() or state.dim() != 4:
        raise ValueError("expected a contiguous CUDA float64 state [nvars, Nr, Ntheta, Nphi]")
    if len(h_vars) != 6 or len(a_vars) != 6:
        raise ValueError("h_vars and a_vars need 6 field indices each")
    nvars, Nr, Nth, Nph = state.shape
    flags = 0
    if theta_filtered is not None:
        if not theta_filtered.is_cuda or theta_filtered.numel() != Nr or theta_filtered.element_size() != 1 \
                or not theta_filtered.is_contiguous():
            raise ValueError("theta_filtered must be a contiguous CUDA byte tensor of Nr flags")
        flags = theta_filtered.data_ptr()
    if theta_filtered is not None and theta_filtered.device != state.device:
        raise ValueError("theta_filtered must be on the state's device")
    hv = (ctypes.c_int * 6)(*[int(k) for k in h_vars])
    av = (ctypes.c_int * 6)(*[int(k) for k in a_vars])
    with torch.cuda.device(state.device):
        if stream is None:
            stream = torch.cuda.current_stream(state.device)
        _check(load().sph_enforce_constraints(state.data_ptr(), nvars, Nr, Nth, Nph, hv, av, int(alpha_var), flags,
                                              float(alpha_bh), _stream_handle(stream)), "sph_enforce_constraints")
    return state
