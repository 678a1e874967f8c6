"""The toy substep loop with the CUDA filter (GPU): the same trajectory as with the oracle as the
filter, and stable at a step several times the axis limit of the unfiltered scheme."""
import math

import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import substep as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


@pytest.mark.parametrize("precision", [0, 2])
def test_cuda_filter_in_the_loop_matches_the_oracle(torch_cuda, precision):
    torch = torch_cuda
    Nth, Nph = 32, 64
    th_lim, ax_lim = S.RotationAdvection(Nth, Nph).cfl_steps()
    dt = 0.5 * th_lim  # ten times the axis limit
    steps = int(round(4 * math.pi / dt))  # two rotations
    u0 = S.blob(Nth, Nph)
    Pg = S.RotationAdvection(Nth, Nph, xp=torch, device="cuda")
    filt = S.plan_filter(Nth, Nph, L=1.0, kind=2, precision=precision)
    ug, peaks = S.run(torch.from_numpy(u0).cuda(), steps, dt, Pg, filt)
    assert filt.plan.sync_status() == 0
    assert max(peaks) <= 1.0 + 1e-12 and peaks[-1] > 0.5
    Pc = S.RotationAdvection(Nth, Nph)
    r = np.array([Nph / 4.0])
    uc, _ = S.run(u0, steps, dt, Pc, lambda u: oracle.filter(u[None, None], [0], [2], [1.0], r, 1.0, 2.0)[0, 0])
    assert np.abs(ug.cpu().numpy() - uc).max() <= 1e-11
