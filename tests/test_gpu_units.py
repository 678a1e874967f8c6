"""Parity of the split launch with the oracle, through the C ABI, on a GB300.

A shell whose theta pass is the identity (exponential or sharp filter with l_max >= Ntheta) changes
only in its active phi rings. A plan with such shells filters them with a kernel over their active
ring pairs (each pair scaled on its own in compensated FP32) after a copy of the shells (out of
place), and runs the shell kernel over the other shells only. Every other test of the plain form
runs through this split too; the cases here pin its own boundaries: every compiled length and the
general one, a lone middle ring (odd Ntheta), plans with no dense shell or no active ring, partial
field ranges, in-place calls, the transpose, and the number of kernels each call enqueues.

Tolerance 1e-13 of the field maximum, as for the other plain-form tests.
"""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

TOL = 1e-13
PRECS = [0, 2]  # SPH_PREC_F64, SPH_PREC_F32X2

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
    return np.array([np.abs(y[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300) for v in range(ref.shape[0])])


def mixed_grid(Nr, Nth, Nph, r_max=40.0):
    """Fields whose shells are all dense (Gaussian; exponential with a small L), mostly sparse
    (exponential and sharp with larger L) or split by radius, with both parities."""
    parity = [0, 1, 0, 1, 0, 1, 0]
    kind = [W.EXP, W.EXP, W.GAUSS, W.SHARP, W.SHARP, W.EXP, W.GAUSS]
    L = [3.0, 12.0, 3.0, 3.0, 0.9, 0.05, 12.0]
    r = np.linspace(0.0, r_max, Nr)
    return W.Grid(Nr, Nth, Nph, parity, kind, L, r)


def sparse_count(g):
    """(dense, sparse) shells of a grid, by the identity-theta criterion."""
    dense = sparse = 0
    for v in range(g.nvars):
        for i in range(g.Nr):
            lm = oracle.lmax(g.r[i], g.dr_min, g.L[v], g.floor)
            if g.kind[v] in (W.EXP, W.SHARP) and not lm < g.Ntheta:
                sparse += 1
            else:
                dense += 1
    return dense, sparse


def run(torch, g, x, prec, inplace=False, fn="apply"):
    from paper_2305_01537_gb300 import Plan
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    n0 = plan.launch_count
    out = getattr(plan, fn)(xd, out=xd if inplace else None)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return out.cpu().numpy(), plan.launch_count - n0, plan


# the compiled lengths, and general ones (transforms of radices 8, 4, 2 and 3 only: other
# lengths run the chunked FP64 kernel, without the split)
@pytest.mark.parametrize("Nth,Nph", [(16, 32), (32, 64), (48, 96), (64, 128), (96, 192), (9, 18), (12, 36)])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("inplace", [False, True])
def test_mixed_plan_all_lengths(torch_cuda, Nth, Nph, prec, inplace):
    g = mixed_grid(10, Nth, Nph)
    dense, sparse = sparse_count(g)
    assert dense > 0 and sparse > 0
    x = W.random_state(g.shape, seed=Nth * 7 + Nph + (100 if inplace else 0))
    ref = oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    y, n, plan = run(torch_cuda, g, x, prec, inplace)
    assert field_errors(y, ref).max() <= TOL
    assert n == (2 if inplace else 3) and plan.launches == 3


@pytest.mark.parametrize("prec", PRECS)
def test_transpose_of_split_plan(torch_cuda, prec):
    g = mixed_grid(9, 32, 64)
    x = W.random_state(g.shape, seed=71)
    ref = oracle.filter_T(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    y, n, _ = run(torch_cuda, g, x, prec, fn="apply_adjoint")
    assert field_errors(y, ref).max() <= TOL and n == 3


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("Nth,Nph,r", [(3, 12, [3.0, 4.0, 5.0, 6.0, 8.0, 11.0]),
                                       (9, 24, [9.0, 10.0, 11.0, 20.0, 40.0, 60.0]),
                                       (27, 96, [27.0, 30.0, 40.0, 47.0, 60.0, 90.0])])
def test_lone_middle_ring(torch_cuda, prec, Nth, Nph, r):
    """Odd Ntheta: the middle ring has no mirror and is filtered alone (paired with a zero row). In
    a shell with an identity theta pass (l_max >= Ntheta) it is active only if Nphi/2 > l_max, so the
    grids have Nphi > 2 Ntheta."""
    g = W.Grid(len(r), Nth, Nph, [0, 1], [W.EXP, W.SHARP], [0.5, 0.5], np.array(r))
    mid = (Nth - 1) // 2
    assert any(oracle.mmax(ri, g.dr_min, 0.5, mid, Nth, g.floor) < Nph / 2 for ri in r)
    x = W.random_state(g.shape, seed=Nth)
    ref = oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    y, n, _ = run(torch_cuda, g, x, prec)
    assert field_errors(y, ref).max() <= TOL
    assert sparse_count(g)[0] == 0 and n == 2  # no dense shell: copy + units


@pytest.mark.parametrize("prec", PRECS)
def test_no_active_ring(torch_cuda, prec):
    """Sharp filter with every cutoff past the grid: the filter is the identity, and a call is a copy
    (out of place) or nothing at all (in place)."""
    g = W.Grid(4, 32, 64, [0, 1], [W.SHARP, W.SHARP], [200.0, 200.0], np.array([50.0, 60.0, 70.0, 80.0]))
    x = W.random_state(g.shape, seed=5)
    y, n, _ = run(torch_cuda, g, x, prec)
    assert np.array_equal(y, x) and n == 1
    y, n, _ = run(torch_cuda, g, x, prec, inplace=True)
    assert np.array_equal(y, x) and n == 0


@pytest.mark.parametrize("prec", PRECS)
def test_host_entry_field_chunks(torch_cuda, prec):
    """The host-buffer call filters field ranges on several streams: each range uses its own part of
    the dense, sparse and unit lists."""
    import torch
    from paper_2305_01537_gb300 import Plan
    g = mixed_grid(12, 32, 64)
    x = W.random_state(g.shape, seed=3)
    ref = oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    plan = Plan.from_grid(g, precision=prec)
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    for _ in range(3):
        oh.zero_()
        plan.apply_host(xh, oh)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        assert field_errors(oh.numpy(), ref).max() <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_f32_input_takes_whole_shells(torch_cuda, prec):
    """FP32 input and output: one shell-kernel launch over every shell, same result within FP32."""
    g = mixed_grid(8, 32, 64)
    x = W.random_state(g.shape, seed=8).astype(np.float32)
    ref = oracle.filter(x.astype(np.float64), g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    y, n, _ = run(torch_cuda, g, x, prec)
    assert field_errors(y.astype(np.float64), ref).max() <= 1e-6 and n == 1


@pytest.mark.parametrize("prec", PRECS)
def test_units_with_scales_apart(torch_cuda, prec):
    """Ring pairs of one shell whose magnitudes differ by up to 2^600: every ring keeps the
    accuracy of its own magnitude (compensated FP32 scales each ring pair by its own power of two,
    where one scale for the whole shell would flush the small rings).

    Reference: these shells have an identity theta pass, so the filter acts ring by ring and
    commutes with a per-ring scale D: F(D x) = D F(x), with F(x) from the oracle on the unscaled
    state. (The oracle applied to D x itself runs the theta round trip with unit multipliers, whose
    rounding carries 1e-16 of the large rings into the small ones.)"""
    g = W.Grid(3, 16, 32, [0], [W.EXP], [4.0], np.array([5.0, 8.0, 12.0]))
    assert sparse_count(g)[0] == 0
    x = W.random_state(g.shape, seed=12)
    j = np.arange(16)
    scale = np.ldexp(1.0, (np.minimum(j, 15 - j) % 4) * 200 - 300)[None, None, :, None]  # mirror rings alike
    ref = oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor) * scale
    y, n, _ = run(torch_cuda, g, x * scale, prec)
    assert n == 2
    for jr in range(16):
        err = np.abs(y[:, :, jr] - ref[:, :, jr]).max() / np.abs(ref[:, :, jr]).max()
        assert err <= TOL, (jr, err)


@pytest.mark.parametrize("prec", PRECS)
def test_same_plan_on_two_streams(torch_cuda, prec):
    """Calls of one split plan on two streams, each forking its copy and units kernels onto the
    plan's side stream: every result is the filter of its own input."""
    import torch
    from paper_2305_01537_gb300 import Plan
    g = mixed_grid(12, 32, 64)
    xs = [W.random_state(g.shape, seed=40 + k) for k in range(4)]
    refs = [oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor) for x in xs]
    plan = Plan.from_grid(g, precision=prec)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    torch.cuda.synchronize()
    for rep in range(3):
        outs = [torch.empty_like(x) for x in xd]
        for k in range(4):
            plan.apply(xd[k], out=outs[k], stream=streams[k % 2])
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        for k in range(4):
            assert field_errors(outs[k].cpu().numpy(), refs[k]).max() <= TOL, (rep, k)


@pytest.mark.parametrize("prec", PRECS)
def test_split_plan_in_cuda_graph(torch_cuda, prec):
    """A split call captured into a CUDA graph (the fork onto the side stream and the join are
    captured as graph edges) and replayed on new inputs."""
    import torch
    from paper_2305_01537_gb300 import Plan
    g = mixed_grid(10, 32, 64)
    plan = Plan.from_grid(g, precision=prec)
    x = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.apply(x, out=y, stream=s)  # warm-up outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.apply(x, out=y, stream=s)
    for seed in (1, 2):
        xh = W.random_state(g.shape, seed=seed)
        x.copy_(torch.from_numpy(xh))
        graph.replay()
        torch.cuda.synchronize()
        ref = oracle.filter(xh, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
        assert field_errors(y.cpu().numpy(), ref).max() <= TOL
