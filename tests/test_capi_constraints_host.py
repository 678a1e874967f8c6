"""Argument validation of sph_enforce_constraints on the host: every rejection happens before any
CUDA call, so it needs no GPU (the state pointer is never dereferenced on the host)."""
import ctypes

import pytest

from paper_2305_01537_gb300.binding import load

EINVAL = 1
FAKE = ctypes.c_void_p(1 << 20)  # never dereferenced: validation fails first


def call(state=FAKE, nvars=13, Nr=2, Nth=3, Nph=4, h=(0, 1, 2, 3, 4, 5), a=(6, 7, 8, 9, 10, 11), alpha=12,
         alpha_bh=0.3):
    hv = (ctypes.c_int * 6)(*h) if h is not None else None
    av = (ctypes.c_int * 6)(*a) if a is not None else None
    return load().sph_enforce_constraints(state, nvars, Nr, Nth, Nph, hv, av, alpha, None, alpha_bh, None)


@pytest.mark.parametrize("kw", [
    dict(state=None), dict(nvars=12), dict(Nr=0), dict(Nth=0), dict(Nph=0), dict(h=None), dict(a=None),
    dict(alpha=13), dict(alpha=-1), dict(h=(0, 1, 2, 3, 4, 4)), dict(a=(6, 7, 8, 9, 10, 0)), dict(alpha=11),
    dict(alpha_bh=float("nan")), dict(alpha_bh=float("inf")), dict(state=ctypes.c_void_p((1 << 20) + 4)),
])
def test_rejections(kw):
    assert call(**kw) == EINVAL
