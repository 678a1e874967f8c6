"""The per-rank step of the angular decomposition on a GB300: plan_slab_filter filters one slab of
whole shells (radii [i0, i1) of a 28-field state) with a CUDA plan built for those radii. The result
must match the oracle on the same slab within 1e-13 of each field's maximum (the plain-form bound),
for a host slab (returned on the host) and a device slab, and a second slab reuses nothing wrongly."""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

TOL = 1e-13

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


def _err(y, ref):
    return max(np.abs(y[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300) for v in range(ref.shape[0]))


@pytest.mark.parametrize("precision", [0, 2])
def test_slab_filter_matches_oracle(torch_cuda, precision):
    torch = torch_cuda
    from paper_2305_01537_gb300.angular import plan_slab_filter
    g = W.grid_28(9, 16, 32)
    x = W.band_limited_state(g, seed=5, mode_max=6, noise=0.1)
    run = plan_slab_filter(g, precision)
    for (i0, i1), on_device in [((2, 7), False), ((0, 2), True), ((2, 7), True)]:
        xs = torch.from_numpy(np.ascontiguousarray(x[:, i0:i1]))
        if on_device:
            xs = xs.cuda()
        y = run(i0, i1, xs)
        torch.cuda.synchronize()
        assert y.device == xs.device
        ref = oracle.filter(x[:, i0:i1], g.parity, g.kind, g.L, g.r[i0:i1], g.dr_min, g.floor)
        assert _err(y.cpu().numpy(), ref) < TOL
