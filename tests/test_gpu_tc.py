"""Parity of the split-precision tensor-core form (SPH_PREC_SPLIT_TC) with the oracle, through the C
ABI (GPU). The form computes only the removed part H x = x - F x from exact BF16 slice products
(six slices per operand) and subtracts it in FP64; its target is 1e-11 in the per-field
normalised max norm (max |y - y_ref| / max |y_ref|), against 1e-13 for the plain form."""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11
TC = 1  # SPH_PREC_SPLIT_TC


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


def oracle_of(g, x, transpose=False):
    f = oracle.filter_T if transpose else oracle.filter
    return f(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)


def sampled_errors(y_of, ref, shells):
    """Sampled shells against the oracle, each normalised by the largest reference value among its
    field's sampled shells (at most the field maximum the full-field measure divides by)."""
    fmax = {v: max(np.abs(ref[n]).max() for n, s in enumerate(shells) if s[0] == v) for v, _ in shells}
    return np.array([np.abs(y_of(v, i) - ref[n]).max() / fmax[v] for n, (v, i) in enumerate(shells)])


@pytest.mark.parametrize("Nr,Nth,Nph", [(3, 4, 8), (4, 8, 16), (3, 16, 32), (2, 12, 40), (3, 32, 24), (2, 5, 74),
                                        (2, 48, 200)])
def test_tiny_and_ragged_grids(torch_cuda, Nr, Nth, Nph):
    """Every field class of the 28-field mix; lengths that are not powers of two, ragged GEMM tiles
    (fewer than 128 vectors, padded K and N) and outputs split over two passes (Nphi = 200)."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(Nr, Nth, Nph)
    x = W.band_limited_state(g, seed=Nr * 100 + Nth, mode_max=3, noise=0.05)
    plan = Plan.from_grid(g, precision=TC)
    xd = torch.from_numpy(x).cuda()
    y = plan.apply(xd).cpu().numpy()
    yt = plan.apply_adjoint(xd).cpu().numpy()
    assert plan.sync_status() == 0
    assert field_errors(y, oracle_of(g, x)).max() <= TOL
    assert field_errors(yt, oracle_of(g, x, True)).max() <= TOL


@pytest.mark.parametrize("Nth,Nph", [(64, 128), (128, 256)])
def test_28_field_mix_headline_shapes(torch_cuda, Nth, Nph):
    """The shell shapes of the 128 x 64 x 128 and 256 x 128 x 256 workloads at radii inside and
    past the cutoff thresholds (many tiles; two shells per tile for Nphi = 128)."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(3, Nth, Nph)
    g.r = np.array([0.5, 7.5, 40.5])
    x = W.band_limited_state(g, seed=77, mode_max=Nph // 8, noise=0.05)
    plan = Plan.from_grid(g, precision=TC)
    xd = torch.from_numpy(x).cuda()
    y = plan.apply(xd).cpu().numpy()
    yt = plan.apply_adjoint(xd).cpu().numpy()
    assert plan.sync_status() == 0
    err = field_errors(y, oracle_of(g, x))
    assert err.max() <= TOL, err
    assert field_errors(yt, oracle_of(g, x, True)).max() <= TOL


def test_in_place_and_random_input(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(4, 16, 32)
    x = W.random_state(g.shape, 12)
    plan = Plan.from_grid(g, precision=TC)
    xd = torch.from_numpy(x).cuda()
    plan.apply(xd, out=xd)
    assert plan.sync_status() == 0
    assert field_errors(xd.cpu().numpy(), oracle_of(g, x)).max() <= TOL


def test_host_entry_and_scaled_fields(torch_cuda):
    """Fields of very different magnitudes (1e-30 .. 1e30): the slicing scale is per vector. The
    host-buffer call runs its field chunks on three streams; repeated, since launches of one plan
    that overlapped would share the kernel's scratch."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(3, 8, 16)
    x = W.band_limited_state(g, seed=5, mode_max=3, noise=0.05)
    x *= np.logspace(-30, 30, 28)[:, None, None, None]
    ref = oracle_of(g, x)
    plan = Plan.from_grid(g, precision=TC)
    xh = torch.from_numpy(x).pin_memory()
    for _ in range(3):
        out = torch.empty_like(xh).pin_memory()
        plan.apply_host(xh, out)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        assert field_errors(out.numpy(), ref).max() <= TOL


def test_same_plan_on_two_streams(torch_cuda):
    """The tensor-core kernel keeps per-CTA scratch in the plan: calls of one plan on two streams
    are chained by the library, so concurrent calls give exactly the single-call results."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(8, 32, 64)
    g.r = np.linspace(0.5, 20.5, 8)
    x1 = torch.from_numpy(W.band_limited_state(g, seed=71, mode_max=6, noise=0.05)).cuda()
    x2 = torch.from_numpy(W.band_limited_state(g, seed=72, mode_max=6, noise=0.05)).cuda()
    plan = Plan.from_grid(g, precision=TC)
    ref1, ref2 = plan.apply(x1), plan.apply(x2)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(10):
        o1, o2 = torch.empty_like(x1), torch.empty_like(x2)
        torch.cuda.synchronize()
        plan.apply(x1, out=o1, stream=s1)
        plan.apply(x2, out=o2, stream=s2)
        torch.cuda.synchronize()
        assert torch.equal(o1, ref1) and torch.equal(o2, ref2)
    assert plan.sync_status() == 0


def test_unsupported_calls(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan, SphFilterError
    g = W.grid_28(2, 8, 16)
    plan = Plan.from_grid(g, precision=TC)
    z = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(SphFilterError):
        plan.apply_tanh(z)
    with pytest.raises(SphFilterError):
        plan.apply(z.float())
    with pytest.raises(SphFilterError):  # vectors longer than 256
        Plan.from_grid(W.grid_28(2, 8, 512), precision=TC)


def test_full_state_256x128x256_sampled(torch_cuda):
    """The 28-field Nr=256, Ntheta=128, Nphi=256 workload at full size, in the launch configuration
    the benchmark times; the oracle checks sampled shells of every field class."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    wl = W.full_state_256x128x256()
    g = wl.grids[0]
    x = wl.state()
    plan = Plan.from_grid(g, precision=TC)
    xd = torch.from_numpy(x).cuda()
    y = plan.apply(xd)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    del xd
    shells = [(v, i) for v in (0, 14, 18, 20, 24, 26) for i in (0, 5, 21, 255)]
    ref = oracle.filter_shells(x, shells, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    err = sampled_errors(lambda v, i: y[v, i].cpu().numpy(), ref, shells)
    assert err.max() <= TOL, shells[int(err.argmax())]


def test_full_state_128x64x128_sampled(torch_cuda):
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    wl = W.full_state_128x64x128()
    g = wl.grids[0]
    x = wl.state()
    plan = Plan.from_grid(g, precision=TC)
    y = plan.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    shells = [(v, i) for v in (0, 13, 14, 19, 23, 25, 27) for i in (0, 3, 17, 127)]
    ref = oracle.filter_shells(x, shells, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    err = sampled_errors(lambda v, i: y[v, i], ref, shells)
    assert err.max() <= TOL, shells[int(err.argmax())]


def test_adjoint_identity(torch_cuda):
    """<F x, y> = <x, F^T y> with both sides from the tensor-core form (Sec. II.C passes are
    symmetric, so F^T runs the phi pass, then the theta pass)."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28(3, 16, 32)
    x = W.random_state(g.shape, 21)
    y = W.random_state(g.shape, 22)
    plan = Plan.from_grid(g, precision=TC)
    fx = plan.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    fty = plan.apply_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    lhs, rhs = float((fx * y).sum()), float((x * fty).sum())
    assert abs(lhs - rhs) <= 1e-11 * np.sqrt((x * x).sum() * (y * y).sum())


def test_batch_and_graph_with_tensor_core_plans(torch_cuda):
    """The batch API and its CUDA-graph replay run tensor-core plans of uneven grids exactly as the
    single-plan calls do (same kernels on the same vectors)."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Batch, Plan
    shapes = [(16, 32, 3), (32, 64, 2), (64, 128, 2), (128, 256, 1)]
    plans, xs = [], []
    for n, (Nth, Nph, Nr) in enumerate(shapes):
        g = W.grid_28(Nr, Nth, Nph)
        g.r = np.linspace(0.5, 40.5, Nr)
        plans.append(Plan.from_grid(g, precision=TC))
        xs.append(torch.from_numpy(W.band_limited_state(g, seed=60 + n, mode_max=4, noise=0.05)).cuda())
    b = Batch(plans)
    outs = [torch.empty_like(x) for x in xs]
    b.apply(xs, outs)
    torch.cuda.synchronize()
    for p, x, o in zip(plans, xs, outs):
        assert torch.equal(o, p.apply(x))
    # three applications per graph launch: in -> out, then out -> out twice
    outs3 = [torch.empty_like(x) for x in xs]
    b.capture(xs, outs3, 3)
    b.launch()
    torch.cuda.synchronize()
    for p, x, o in zip(plans, xs, outs3):
        ref = p.apply(p.apply(p.apply(x)))
        assert torch.equal(o, ref)
    assert all(p.sync_status() == 0 for p in plans)
