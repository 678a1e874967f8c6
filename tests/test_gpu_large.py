"""Parity of the cluster-pair kernel (shells of Ntheta x Nphi = 128 x 256, too large for one CTA's
shared memory) with the oracle, through the C ABI (GPU). Same error measure and 1e-13 tolerance as
the other plain-form tests."""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


def field_errors(y, ref):
    return np.array([np.abs(y[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300) for v in range(ref.shape[0])])


@pytest.mark.parametrize("prec", [0, 2])
def test_cluster_shells_all_classes(torch_cuda, prec):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(3, 128, 256)
    g.r = np.array([0.5, 10.5, 100.5])
    x = W.band_limited_state(g, seed=31, mode_max=12, noise=0.05)
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(x).cuda()
    y = plan.apply(xd).cpu().numpy()
    yt = plan.apply_adjoint(xd).cpu().numpy()
    assert plan.sync_status() == 0
    args = (g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    assert field_errors(y, oracle.filter(x, *args)).max() <= TOL
    assert field_errors(yt, oracle.filter_T(x, *args)).max() <= TOL


@pytest.mark.parametrize("prec", [0, 2])
def test_cluster_tanh_maps_fp32(torch_cuda, prec):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    p, k, L = W.field_mix_8()
    g = W.Grid(2, 128, 256, p, k, L, np.array([0.5, 30.5]))
    z = W.random_state(g.shape, 4)
    gr = W.random_state(g.shape, 5)
    plan = Plan.from_grid(g, precision=prec)
    zd, gd = torch.from_numpy(z).cuda(), torch.from_numpy(gr).cuda()
    args = (g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    y = plan.apply_tanh(zd).cpu().numpy()
    assert field_errors(y, oracle.filter(np.tanh(z), *args)).max() <= TOL
    d = plan.apply_adjoint_tanh(gd, zd).cpu().numpy()
    assert field_errors(d, (1 - np.tanh(z) ** 2) * oracle.filter_T(gr, *args)).max() <= TOL
    y32 = plan.apply(zd.float()).cpu().numpy().astype(np.float64)
    assert field_errors(y32, oracle.filter(z.astype(np.float32).astype(np.float64), *args)).max() <= 2e-6


@pytest.mark.parametrize("prec", [0, 2])
def test_full_state_256x128x256_sampled(torch_cuda, prec):
    """The 28-field Nr=256, Ntheta=128, Nphi=256 workload (3.76 GB of FP64 I/O) at full size; the
    oracle checks a sample of shells of every field class at radii inside and past the thresholds."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    wl = W.full_state_256x128x256()
    g = wl.grids[0]
    x = wl.state()
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(x).cuda()
    y = plan.apply(xd)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    del xd
    shells = [(v, i) for v in (0, 14, 18, 20, 24, 26) for i in (0, 5, 21, 255)]
    ref = oracle.filter_shells(x, shells, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    got = np.stack([y[v, i].cpu().numpy() for (v, i) in shells])
    err = np.array([np.abs(got[n] - ref[n]).max() / np.abs(ref[n]).max() for n in range(len(shells))])
    assert err.max() <= TOL, shells[int(err.argmax())]
