"""Differentiable chain loss = sum w * (F o tanh o ... o tanh o F x)^2 through the C ABI (GPU).

Checks the gradient of the fused adjoint kernels against (1) a gradient built from the oracle alone
(its forward filter and its explicit transpose, the chain rule written out in numpy), (2) central
finite differences (h = 1e-6, FP64) along random directions, (3) the adjoint identity
<F x, y> = <x, F^T y>, and (4) bitwise equality of the checkpointed and the stored-activation
gradients. FP64 and FP32 storage.
"""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


def oracle_chain_grad(x, w, g, n):
    """Loss and gradient of sum w y^2 from the oracle's F and F^T with the chain rule in numpy."""
    F = lambda t: oracle.filter(t, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    FT = lambda t: oracle.filter_T(t, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    pre = []  # inputs of the tanh maps
    y = F(x)
    for _ in range(n - 1):
        pre.append(y)
        y = F(np.tanh(y))
    loss = float((w * y * y).sum())
    gy = 2.0 * w * y
    for z in reversed(pre):
        gy = (1.0 - np.tanh(z) ** 2) * FT(gy)
    return loss, FT(gy)


def small_chain_grid():
    p, k, L = W.field_mix_8()
    return W.Grid(6, 16, 32, p, k, L, np.array([0.5, 1.5, 2.5, 4.5, 8.5, 16.5]))


@pytest.mark.parametrize("prec", [0, 2])
def test_chain_gradient_matches_oracle(torch_cuda, prec):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    from paper_2305_01537_gb300.autograd import chain_loss
    g = small_chain_grid()
    x = W.band_limited_state(g, seed=9, mode_max=4, noise=0.05) * 0.1
    w = W.chain_weights(g)
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    loss = chain_loss(xd, plan, torch.from_numpy(w).cuda(), 8)
    loss.backward()
    ref_loss, ref_grad = oracle_chain_grad(x, w, g, 8)
    assert abs(loss.item() - ref_loss) <= 1e-12 * abs(ref_loss)
    gr = xd.grad.cpu().numpy()
    assert np.abs(gr - ref_grad).max() <= 1e-12 * np.abs(ref_grad).max()


def test_chain_gradient_finite_differences(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    from paper_2305_01537_gb300.autograd import chain_loss
    g = small_chain_grid()
    x = W.band_limited_state(g, seed=19, mode_max=4, noise=0.05) * 0.1
    w = torch.from_numpy(W.chain_weights(g)).cuda()
    plan = Plan.from_grid(g)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    chain_loss(xd, plan, w, 8).backward()
    grad = xd.grad.detach()
    rng = np.random.default_rng(5)
    h = 1e-6
    with torch.no_grad():
        for _ in range(16):
            d = torch.from_numpy(rng.standard_normal(g.shape)).cuda()
            lp = chain_loss(xd + h * d, plan, w, 8).item()
            lm = chain_loss(xd - h * d, plan, w, 8).item()
            fd = (lp - lm) / (2 * h)
            an = float((grad * d).sum())
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_adjoint_identity(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(8, 32, 64)
    plan = Plan.from_grid(g)
    x = torch.from_numpy(W.random_state(g.shape, 1)).cuda()
    y = torch.from_numpy(W.random_state(g.shape, 2)).cuda()
    lhs = float((plan.apply(x) * y).sum())
    rhs = float((x * plan.apply_adjoint(y)).sum())
    assert abs(lhs - rhs) <= 1e-13 * float(x.norm() * y.norm())


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_checkpointed_gradient_bitwise_equal(torch_cuda, dtype):
    """The 8-field Nr=128, Ntheta=64, Nphi=128 chain workload: recomputed activations give the same
    gradient bit for bit (every kernel is deterministic)."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    from paper_2305_01537_gb300.autograd import chain_loss
    wl = W.chain_8field()
    g = wl.grids[0]
    td = torch.float64 if dtype == "f64" else torch.float32
    x = torch.from_numpy(wl.state() * 0.1).to("cuda", td)
    w = torch.from_numpy(W.chain_weights(g)).to("cuda", td)
    plan = Plan.from_grid(g)
    grads = []
    for ck in (0, 1, 3):
        xd = x.clone().requires_grad_(True)
        chain_loss(xd, plan, w, 8, checkpoint_every=ck).backward()
        grads.append(xd.grad.clone())
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])


def test_fp32_chain_gradient(torch_cuda):
    """FP32 storage of the chain: gradient within FP32 rounding of the FP64 oracle gradient."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    from paper_2305_01537_gb300.autograd import chain_loss
    g = small_chain_grid()
    x = W.band_limited_state(g, seed=29, mode_max=4, noise=0.05) * 0.1
    w = W.chain_weights(g)
    plan = Plan.from_grid(g)
    xd = torch.from_numpy(x).to("cuda", torch.float32).requires_grad_(True)
    chain_loss(xd, plan, torch.from_numpy(w).to("cuda", torch.float32), 8).backward()
    _, ref = oracle_chain_grad(x.astype(np.float32).astype(np.float64), w.astype(np.float32).astype(np.float64), g, 8)
    gr = xd.grad.double().cpu().numpy()
    assert np.abs(gr - ref).max() <= 1e-5 * np.abs(ref).max()
