"""Host-side checks of the C ABI (CPU only): the library loads, exports every function that
include/*.h declares, and rejects invalid arguments before touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_01537_gb300 import build as B
    B.build()
    from paper_2305_01537_gb300 import binding
    return binding.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sph_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sph_filter_plan_create", "sph_filter_apply", "sph_filter_apply_adjoint",
                     "sph_filter_plan_destroy", "sph_filter_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2305_01537_gb300 import binding
    assert set(binding.EXPORTED) == set(declared_functions())


def test_status_strings(lib):
    from paper_2305_01537_gb300 import binding
    assert binding.sph_filter_status_string(0) == "ok"
    assert "overlap" in binding.sph_filter_status_string(6)
    assert binding.sph_filter_status_string(99) == "unknown status"


def _create(lib, Nr=2, Nth=4, Nph=8, parity=(0,), kind=(0,), L=(3.0,), r=None, dr_min=1.0, floor=2.0,
            precision=0, eps=1e-12):
    from paper_2305_01537_gb300 import binding
    nv = len(parity)
    par = np.asarray(parity, dtype=np.int32)
    kd = np.asarray(kind, dtype=np.int32)
    Ls = np.asarray(L, dtype=np.float64)
    rs = np.asarray(r if r is not None else np.arange(Nr) + 0.5, dtype=np.float64)
    prm = binding.sph_cutoff_params(rs.ctypes.data, dr_min, Ls.ctypes.data, kd.ctypes.data, floor, precision, eps)
    h = ctypes.c_void_p()
    st = lib.sph_filter_plan_create(ctypes.byref(h), Nr, Nth, Nph, nv, par.ctypes.data, ctypes.byref(prm))
    if st == 0:
        lib.sph_filter_plan_destroy(h)
    return st


def test_plan_create_rejects_invalid_arguments(lib):
    EINVAL = 1
    assert _create(lib, Nph=7) == EINVAL          # odd Nphi
    assert _create(lib, Nph=0) == EINVAL
    assert _create(lib, Nr=0) == EINVAL
    assert _create(lib, Nth=0) == EINVAL
    assert _create(lib, parity=(2,)) == EINVAL
    assert _create(lib, kind=(4,)) == EINVAL
    assert _create(lib, kind=(-1,)) == EINVAL
    assert _create(lib, kind=(3,), eps=-1.0) == EINVAL         # hybrid field: eps >= 0 and finite
    assert _create(lib, kind=(3,), eps=float("nan")) == EINVAL
    assert _create(lib, kind=(3,), eps=float("inf")) == EINVAL
    assert _create(lib, L=(0.0,)) == EINVAL
    assert _create(lib, r=[0.5, -1.0]) == EINVAL
    assert _create(lib, dr_min=0.0) == EINVAL
    assert _create(lib, floor=-1.0) == EINVAL
    assert _create(lib, precision=7) == EINVAL
    h = ctypes.c_void_p()
    assert lib.sph_filter_plan_create(ctypes.byref(h), 2, 4, 8, 1, None, None) == EINVAL
    assert lib.sph_filter_plan_create(None, 2, 4, 8, 1, None, None) == EINVAL


def test_hybrid_plans_the_tensor_core_form_cannot_run(lib):
    """The split-precision tensor-core form has no per-circle filter switch: a hybrid field there is
    rejected before any device work (SPH_EUNSUPPORTED)."""
    assert _create(lib, kind=(0, 3), parity=(0, 1), L=(3.0, 12.0), precision=1) == 4


def test_spectral_form_rejects_what_it_cannot_run(lib):
    """The spectral form (precision 3) pairs rows 2n and 2n + 1 of every mode and filters whole
    modes: odd Ntheta and hybrid fields are rejected before any device work (SPH_EUNSUPPORTED)."""
    assert _create(lib, Nth=5, Nph=10, precision=3) == 4
    assert _create(lib, kind=(0, 3), parity=(0, 1), L=(3.0, 12.0), precision=3) == 4


def test_calls_on_null_plan_are_rejected(lib):
    assert lib.sph_filter_apply(None, None, None, None) == 1
    assert lib.sph_filter_apply_adjoint(None, None, None, None) == 1
    assert lib.sph_filter_plan_points(None) == 0
    lib.sph_filter_plan_destroy(None)  # no-op


def test_no_cpu_fallback_without_a_device(lib):
    """On a machine without a GPU a valid plan cannot be created: the library reports a CUDA error
    instead of computing anything on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _create(lib) == 3  # SPH_ECUDA
