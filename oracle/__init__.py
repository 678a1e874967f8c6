"""Oracle for the double FFT filter (arXiv:2305.01537, Sec. II.C "Filtering algorithms").

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline
leg are the only callers allowed. The product path never imports this module, and this module
imports nothing from the product package.

The arithmetic lives in ``sph_oracle.c`` (plain C, naive O(N^2) DFTs, FP64). The same source
compiled with ``-DORACLE_LONG_DOUBLE`` gives an extended-precision copy used only to bound the
oracle's own rounding error. This file builds both with gcc and marshals numpy arrays. The
algebraic-constraint map applied after filtering (same section) is ``oracle.constraints`` (numpy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIBS = {"f64": os.path.join(_HERE, "liboracle_f64.so"), "ld": os.path.join(_HERE, "liboracle_ld.so")}
_lock = threading.Lock()
_loaded: dict = {}

KIND_EXP, KIND_GAUSS, KIND_SHARP, KIND_HYBRID = 0, 1, 2, 3


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (OpenMP over shells; no fast-math, no FMA contraction)."""
    for variant, out in _LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC,
               "-o", out + ".tmp", "-lm"]
        if variant == "ld":
            cmd.insert(1, "-DORACLE_LONG_DOUBLE")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


def _lib(variant: str = "f64"):
    with _lock:
        if variant not in _loaded:
            build()
            lib = ctypes.CDLL(_LIBS[variant])
            pre = "oracle_" if variant == "f64" else "oracle_ld_"
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            for name in ("filter", "filter_T"):
                fn = getattr(lib, pre + name)
                fn.argtypes = [I, I, I, I, P, P, P, P, D, D, D, P, P]
                fn.restype = I
            fn = getattr(lib, pre + "single_pass")
            fn.argtypes = [I, I, I, I, P, P, P, P, D, D, D, P, P, I]
            fn.restype = I
            getattr(lib, pre + "detect").argtypes = [I, I, I, D, P, P, P]
            getattr(lib, pre + "detect").restype = I
            getattr(lib, pre + "jameson_fires").argtypes = [D, D, D, D]
            getattr(lib, pre + "jameson_fires").restype = I
            getattr(lib, pre + "filter_value").argtypes = [I, D, D]
            getattr(lib, pre + "filter_value").restype = D
            getattr(lib, pre + "lmax").argtypes = [D, D, D, D]
            getattr(lib, pre + "lmax").restype = D
            getattr(lib, pre + "mmax").argtypes = [D, D, D, D, I, I]
            getattr(lib, pre + "mmax").restype = D
            getattr(lib, pre + "max_threads").restype = I
            getattr(lib, pre + "set_threads").argtypes = [I]
            _loaded[variant] = (lib, pre)
        return _loaded[variant]


def _prep(x, parity, kind, L, r):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 4:
        raise ValueError("state must be [nvars][Nr][Ntheta][Nphi]")
    nvars, Nr, Nth, Nph = x.shape
    parity = np.ascontiguousarray(parity, dtype=np.int32)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    if parity.shape != (nvars,) or kind.shape != (nvars,) or L.shape != (nvars,) or r.shape != (Nr,):
        raise ValueError("parity/kind/L must have nvars entries and r must have Nr entries")
    return x, parity, kind, L, r


def _call(name, x, parity, kind, L, r, dr_min, floor, variant, eps, extra=()):
    x, parity, kind, L, r = _prep(x, parity, kind, L, r)
    lib, pre = _lib(variant)
    out = np.empty_like(x)
    nvars, Nr, Nth, Nph = x.shape
    rc = getattr(lib, pre + name)(Nr, Nth, Nph, nvars, parity.ctypes.data, kind.ctypes.data,
                                  L.ctypes.data, r.ctypes.data, float(dr_min), float(floor), float(eps),
                                  x.ctypes.data, out.ctypes.data, *extra)
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments of {name}")
    return out


def filter(x, parity, kind, L, r, dr_min=1.0, floor=2.0, variant="f64", eps=0.0):
    """The double filter F: theta pass on the double-covered circles, then phi pass on the rings.
    eps: the epsilon of Jameson's detector for hybrid fields (kind 3)."""
    return _call("filter", x, parity, kind, L, r, dr_min, floor, variant, eps)


def filter_T(x, parity, kind, L, r, dr_min=1.0, floor=2.0, variant="f64", eps=0.0):
    """The transpose F^T: phi pass, then theta pass (each pass is real symmetric). Not defined for
    hybrid fields (the switch is nonlinear)."""
    return _call("filter_T", x, parity, kind, L, r, dr_min, floor, variant, eps)


def theta_pass(x, parity, kind, L, r, dr_min=1.0, floor=2.0, variant="f64", eps=0.0):
    return _call("single_pass", x, parity, kind, L, r, dr_min, floor, variant, eps, (1,))


def phi_pass(x, parity, kind, L, r, dr_min=1.0, floor=2.0, variant="f64", eps=0.0):
    return _call("single_pass", x, parity, kind, L, r, dr_min, floor, variant, eps, (2,))


def detect(shell, parity: int, eps: float):
    """Jameson detector flags of one shell [Ntheta, Nphi] (Sec. II.C hybrid filter): (circ, ring),
    circ[k] for the theta circles k < Nphi/2, ring[j] for the phi rings, as bool arrays."""
    shell = np.ascontiguousarray(shell, dtype=np.float64)
    Nth, Nph = shell.shape
    circ = np.zeros(Nph // 2, dtype=np.uint8)
    ring = np.zeros(Nth, dtype=np.uint8)
    lib, pre = _lib("f64")
    rc = getattr(lib, pre + "detect")(Nth, Nph, int(parity), float(eps), shell.ctypes.data, circ.ctypes.data,
                                      ring.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments of detect")
    return circ.astype(bool), ring.astype(bool)


def jameson_fires(a: float, b: float, c: float, eps: float) -> bool:
    """sigma >= 0.95 for one cell u_i = b with neighbours a, c."""
    lib, pre = _lib("f64")
    return bool(getattr(lib, pre + "jameson_fires")(float(a), float(b), float(c), float(eps)))


def filter_value(kind: int, l: float, lmax: float, variant="f64") -> float:
    lib, pre = _lib(variant)
    return getattr(lib, pre + "filter_value")(int(kind), float(l), float(lmax))


def lmax(r: float, dr_min: float, L: float, floor: float = 2.0) -> float:
    lib, pre = _lib("f64")
    return getattr(lib, pre + "lmax")(float(r), float(dr_min), float(L), float(floor))


def mmax(r: float, dr_min: float, L: float, j: int, Nth: int, floor: float = 2.0) -> float:
    lib, pre = _lib("f64")
    return getattr(lib, pre + "mmax")(float(r), float(dr_min), float(L), float(floor), int(j), int(Nth))


def max_threads() -> int:
    lib, pre = _lib("f64")
    return getattr(lib, pre + "max_threads")()


def set_threads(n: int) -> None:
    for v in ("f64",):
        lib, pre = _lib(v)
        getattr(lib, pre + "set_threads")(int(n))


def filter_shells(x, shells, parity, kind, L, r, dr_min=1.0, floor=2.0, transpose=False, eps=0.0):
    """Filter only the listed (v, i) shells of a state; returns an array [len(shells), Ntheta, Nphi].

    Each shell is independent, so this is the oracle evaluated one shell at a time: used to check
    sampled outputs of workloads too large for the full oracle."""
    x = np.asarray(x)
    parity = np.asarray(parity)
    kind = np.asarray(kind)
    L = np.asarray(L)
    r = np.asarray(r)
    out = []
    fn = filter_T if transpose else filter
    for (v, i) in shells:
        s = np.ascontiguousarray(x[v, i][None, None], dtype=np.float64)
        out.append(fn(s, parity[v:v + 1], kind[v:v + 1], L[v:v + 1], r[i:i + 1], dr_min, floor, eps=eps)[0, 0])
    return np.stack(out)
