"""Parity of the spectral form (SPH_PREC_SPECTRAL, FP64) with the oracle, through the C ABI, on a
GB300.

The spectral form computes the same filter as the plain form (Sec. II.C, theta then phi), composed
differently: one phi transform per ring, per azimuthal mode m the theta filter of the mode's even
or odd extension as a cosine/sine transform pair through a complex FFT of length Ntheta, the phi
multiply, one inverse phi transform. The oracle is the same naive DFT filter as for the plain form;
the tolerance is the plain form's, 1e-13 of each field's maximum (the form has a few more roundings
per value than the plain FP64 form, of the same 1.1e-16 size).
"""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

TOL = 1e-13
SPECTRAL = 3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


def field_errors(y, ref):
    nv = ref.shape[0]
    return np.array([np.abs(y[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300) for v in range(nv)])


def args_of(g):
    return (g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)


def run(torch, g, x, fn="apply", **kw):
    from paper_2305_01537_gb300 import Plan
    plan = Plan.from_grid(g, precision=SPECTRAL)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = getattr(plan, fn)(xd, **kw)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return y.cpu().numpy()


def test_single_field_workload(torch_cuda):
    wl = W.single_field()
    g = wl.grids[0]
    x = wl.state()
    assert field_errors(run(torch_cuda, g, x), oracle.filter(x, *args_of(g))).max() <= TOL


@pytest.mark.parametrize("Nth,Nph", [(2, 4), (4, 8), (6, 12), (8, 4), (8, 16), (12, 24), (16, 32), (24, 48),
                                     (32, 64), (48, 96), (6, 32), (16, 12)])
def test_small_and_ragged_grids(torch_cuda, Nth, Nph):
    """Every kind and parity (odd and even extensions of every mode), radii from the origin (the
    floor) to past the identity threshold (shells without a theta pass take the phi pass alone);
    transform lengths with radix 2, 3, 4 and 8 stages, 2 Ntheta both equal to and different from
    Nphi."""
    parity = [0, 1, 0, 1, 0, 1]
    kind = [0, 0, 1, 1, 2, 2]
    L = [0.7, 1.3, 2.0, 0.5, 0.9, 1.1]
    r = np.array([0.0, 0.3, 1.1, 2.6, 7.0, 40.0])
    g = W.Grid(len(r), Nth, Nph, parity, kind, L, r)
    x = W.random_state(g.shape, seed=Nth * 1000 + Nph + 7)
    y = run(torch_cuda, g, x)
    assert field_errors(y, oracle.filter(x, *args_of(g))).max() <= TOL
    yt = run(torch_cuda, g, x, fn="apply_adjoint")
    assert field_errors(yt, oracle.filter_T(x, *args_of(g))).max() <= TOL


def test_band_limited_input_passes_and_parity_mix(torch_cuda):
    """A state of low (l, m) modes of both parities passes the exponential filter unchanged far
    from the origin; near it the filter acts; both match the oracle."""
    wl = W.single_field()
    g0 = wl.grids[0]
    g = W.Grid(g0.Nr, g0.Ntheta, g0.Nphi, [0, 1], [0, 1], [3.0, 12.0])
    x = W.random_state(g.shape, seed=5)
    assert field_errors(run(torch_cuda, g, x), oracle.filter(x, *args_of(g))).max() <= TOL


def test_in_place_and_transpose_28_fields(torch_cuda):
    """The 28-field mix on 24 radii of a 64 x 128 shell (the compiled 128-point form): out of place,
    in place (out = in) and the transpose."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    p, k, L = W.field_mix_28()
    r = np.arange(24) * 5.3 + 0.5
    g = W.Grid(24, 64, 128, p, k, L, r)
    x = W.random_state(g.shape, seed=11)
    ref = oracle.filter(x, *args_of(g))
    assert field_errors(run(torch, g, x), ref).max() <= TOL
    plan = Plan.from_grid(g, precision=SPECTRAL)
    xd = torch.from_numpy(x.copy()).cuda()
    plan.apply(xd, out=xd)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    assert field_errors(xd.cpu().numpy(), ref).max() <= TOL
    yt = run(torch, g, x, fn="apply_adjoint")
    assert field_errors(yt, oracle.filter_T(x, *args_of(g))).max() <= TOL


def test_full_state_128x64x128_sampled(torch_cuda):
    """The 28-field Nr = 128, Ntheta = 64, Nphi = 128 workload at full size; the oracle checks a
    sample of shells of every field class at radii inside and past the thresholds."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    wl = W.full_state_128x64x128()
    g = wl.grids[0]
    x = wl.state()
    plan = Plan.from_grid(g, precision=SPECTRAL)
    xd = torch.from_numpy(x).cuda()
    y = plan.apply(xd)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    shells = [(v, i) for v in (0, 14, 18, 20, 24, 26) for i in (0, 3, 21, 127)]
    ref = oracle.filter_shells(x, shells, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    got = np.stack([y[v, i].cpu().numpy() for (v, i) in shells])
    for n, (v, i) in enumerate(shells):
        scale = max(np.abs(ref[n]).max(), 1e-300)
        assert np.abs(got[n] - ref[n]).max() / scale <= TOL, (v, i)


def test_matches_the_plain_form(torch_cuda):
    """Two compositions of one filter: the spectral and the plain FP64 form agree to rounding."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    p, k, L = W.field_mix_8()
    g = W.Grid(6, 32, 64, p, k, L, np.array([0.0, 0.7, 2.5, 6.0, 12.0, 60.0]))
    x = W.random_state(g.shape, seed=3)
    xd = torch.from_numpy(x).cuda()
    ys = Plan.from_grid(g, precision=SPECTRAL).apply(xd).cpu().numpy()
    yp = Plan.from_grid(g, precision=0).apply(xd).cpu().numpy()
    assert field_errors(ys, yp).max() <= TOL


def test_shapes_the_form_cannot_run(torch_cuda):
    """Odd Ntheta, hybrid fields and shells larger than one CTA are rejected (SPH_EUNSUPPORTED),
    not approximated."""
    from paper_2305_01537_gb300 import Plan, SphFilterError
    for g in (W.Grid(2, 5, 10, [0], [0], [3.0]), W.Grid(2, 8, 16, [0], [3], [3.0]),
              W.Grid(2, 128, 256, [0], [0], [3.0])):
        with pytest.raises(SphFilterError) as e:
            Plan.from_grid(g, precision=SPECTRAL)
        assert e.value.status == 4


@pytest.mark.parametrize("prec", [0, 2, 1, SPECTRAL])
def test_repeated_applications_are_identical(torch_cuda, prec):
    """Every form, on the full 28 x 128 x 64 x 128 state: repeated applications into outputs filled
    with NaN give bit-identical results (a race inside a kernel shows up here as a few shells that
    differ from one run to the next), and every 8th radius of every field matches the oracle."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    wl = W.full_state_128x64x128()
    g = wl.grids[0]
    x = wl.state()
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(x).cuda()
    first = None
    for _ in range(4):
        y = torch.full_like(xd, float("nan"))
        plan.apply(xd, out=y)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        if first is None:
            first = y
        else:
            assert torch.equal(y, first)
    idx = np.arange(0, g.Nr, 8)
    ref = oracle.filter(np.ascontiguousarray(x[:, idx]), g.parity, g.kind, g.L, g.r[idx], g.dr_min, g.floor)
    got = first[:, idx].cpu().numpy()
    tol = 1e-11 if prec == 1 else TOL
    assert field_errors(got, ref).max() <= tol


def test_tanh_maps(torch_cuda):
    """The fused chain steps F(tanh z) and (1 - tanh(z)^2) F^T g in the spectral form, on a grid
    with shells of both kinds (the split launch's spectral shell kernel, copy and units kernels)."""
    from paper_2305_01537_gb300 import Plan
    torch = torch_cuda
    wl = W.chain_8field()
    g = W.Grid(6, 16, 32, wl.grids[0].parity, wl.grids[0].kind, wl.grids[0].L)
    z = W.random_state(g.shape, 3)
    gr = W.random_state(g.shape, 4)
    plan = Plan.from_grid(g, precision=SPECTRAL)
    zd, gd = torch.from_numpy(z).cuda(), torch.from_numpy(gr).cuda()
    y = plan.apply_tanh(zd).cpu().numpy()
    assert field_errors(y, oracle.filter(np.tanh(z), *args_of(g))).max() <= TOL
    d = plan.apply_adjoint_tanh(gd, zd).cpu().numpy()
    ref = (1 - np.tanh(z) ** 2) * oracle.filter_T(gr, *args_of(g))
    assert field_errors(d, ref).max() <= TOL
