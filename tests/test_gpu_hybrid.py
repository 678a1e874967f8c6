"""Parity of the hybrid filter (SPH_FILTER_HYBRID: exponential, or Gaussian where Jameson's shock
detector fires, Sec. II.C) with the oracle, through the C ABI, on a GB300, for the FP64 and the
compensated FP32 precisions.

The detector's decisions are integers decided by floating point: the kernel screens sigma in FP32
and decides every cell within 4e-6 of the threshold (and every cell with a subnormal input) with
the same FP64 expression as the oracle, so the choices must agree exactly. A wrong choice moves
the filtered ring or circle by the difference between the Gaussian and the exponential filter
(1e-6 of the ring's values or more), far above the 1e-13 tolerance of the plain form.
"""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

TOL = 1e-13
PRECS = [0, 2]  # SPH_PREC_F64, SPH_PREC_F32X2
HYB, EXP, GAUSS = 3, 0, 1

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


def oracle_of(g, x):
    return oracle.filter(x, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor, eps=g.eps)


def apply(torch, g, x, prec):
    from paper_2305_01537_gb300 import Plan
    plan = Plan.from_grid(g, precision=prec)
    y = plan.apply(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return y.cpu().numpy()


def star_case(Nr, Nth, Nph, seed=None):
    """Shells from r = 10.5 (inside the star's radii) to 40.5 (outside; the exponential filter is
    the identity there except near the poles); the star's surface crosses r = 5 .. 35."""
    g = W.grid_28_hybrid(Nr, Nth, Nph)
    g.r = np.linspace(10.5, 40.5, Nr)
    x = W.star_state(g, seed=Nr * 100 + Nth if seed is None else seed, centre_r=20.0, radius=15.0)
    return g, x


def fired(g, x):
    """Share of circles and rings whose detector fires, over the hybrid fields (oracle)."""
    c = r = tc = tr = 0
    for v in range(g.nvars):
        if g.kind[v] != HYB:
            continue
        for i in range(g.Nr):
            circ, ring = oracle.detect(x[v, i], g.parity[v], g.eps)
            c, r, tc, tr = c + circ.sum(), r + ring.sum(), tc + circ.size, tr + ring.size
    return c / max(tc, 1), r / max(tr, 1)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("Nr,Nth,Nph", [(3, 4, 8), (2, 3, 6), (4, 8, 16), (3, 6, 12), (2, 9, 54), (2, 12, 48),
                                        (2, 24, 36), (3, 16, 32), (3, 32, 64), (2, 48, 96), (2, 64, 128),
                                        (2, 96, 192), (2, 128, 256)])
def test_star_state_all_lengths(torch_cuda, Nr, Nth, Nph, prec):
    """The 28-field mix with hybrid matter fields on the star state: tiny and ragged shapes (a lone
    circle when Nphi/2 is odd, a lone middle ring when Ntheta is odd), every compiled length, and
    128 x 256 shells (a CTA pair per shell)."""
    g, x = star_case(Nr, Nth, Nph)
    y = apply(torch_cuda, g, x, prec)
    err = field_errors(y, oracle_of(g, x))
    assert err.max() <= TOL, (err.argmax(), err.max())


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_circle_pairs_and_mirror_rings(torch_cuda, prec):
    """Spikes placed so that in one circle pair (2b, 2b+1) only one circle fires and in one mirror
    ring pair (j, Ntheta-1-j) only one ring fires: both take the exact split multiply. One field
    even, one odd; radii where the exponential filter is the identity and where it is not."""
    Nth, Nph = 16, 32
    g = W.Grid(3, Nth, Nph, [0, 1], [HYB, HYB], [3.0, 3.0], r=np.array([0.5, 2.5, 40.5]))
    x = W.few_mode_state(g, seed=12, nmodes=5, mode_max=4, noise=0.0)
    x[0] += 4.0
    # a spike fires its ring and circle when it is some 40 times its neighbours (sigma = 2s/(4a + 2s))
    x[:, :, 5, 6] += 1000.0   # ring 5 (mirror 10) and circle 6 (pair 6, 7) fire
    x[:, 1, 12, 21] -= 1000.0  # on shell 1 also ring 12 (mirror 3) and circle 21 - 16 = 5 (pair 4, 5)
    for v in range(2):
        for i in range(3):
            circ, ring = oracle.detect(x[v, i], g.parity[v], g.eps)
            assert circ[6] and not circ[7] and ring[5] and not ring[Nth - 1 - 5]
    y = apply(torch_cuda, g, x, prec)
    assert field_errors(y, oracle_of(g, x)).max() <= TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("Nth,Nph", [(12, 24), (16, 32), (32, 64), (64, 128), (128, 256)])
def test_decisions_inside_the_screening_band(torch_cuda, prec, Nth, Nph):
    """Cells whose sigma lies within 1e-7 of 0.95, on both sides, in rings and in circles: the
    kernel must take the exact FP64 decision there. A ring (1, x, 1, 1, x, 1, ...) has sigma =
    (1 - x) / (1 + x) at its x cells and about 1/3 elsewhere, so x near 1/39 decides it. Nphi a
    multiple of 32 takes the kernel's column walk, whose undecided cells send the shell to the
    cell-by-cell pass; Nphi = 24 takes that pass directly."""
    rng = np.random.default_rng(3)
    Nr = 6
    g = W.Grid(Nr, Nth, Nph, [0], [HYB], [2.0], r=np.linspace(0.5, 30.5, Nr), eps=0.0)
    x = np.ones(g.shape)
    x0 = 1.0 / 39.0
    for i in range(Nr):
        for j in range(Nth):
            # phi rings: x cells at k = 1 mod 3
            d = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-15, -7)
            x[0, i, j, 1::3] = x0 * (1.0 + d)
        # theta circles: column k = 2 gets the pattern along theta (rows 1, 4, 7, 10)
        d = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-15, -7)
        x[0, i, 1::3, 2] = x0 * (1.0 + d)
    fc, fr = fired(g, x)
    assert 0.0 < fr < 1.0 and 0.0 < fc < 1.0  # both decisions occur
    y = apply(torch_cuda, g, x, prec)
    assert field_errors(y, oracle_of(g, x)).max() <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_cta_pair_block_edges(torch_cuda, prec):
    """128 x 256 shells run on a CTA pair: rank r holds the meridian blocks r and r + 2 (64 columns
    each), so a ring cell at a block edge has its phi neighbour on the other CTA. Each marked row
    holds a single dip (1, 0.02, 1) (sigma 0.96) at one edge column, and nothing else in the ring
    reaches 0.95: the ring fires only if the neighbour read across the pair is right."""
    Nth, Nph = 128, 256
    g = W.Grid(2, Nth, Nph, [0, 1], [HYB, HYB], [3.0, 3.0], r=np.array([20.5, 60.5]))
    x = np.ones(g.shape) + 1e-3 * W.few_mode_state(g, seed=41, nmodes=3, mode_max=3, noise=0.0)
    edges = {5: 63, 20: 64, 35: 127, 50: 128, 70: 191, 85: 192, 100: 255, 115: 0}
    for j, c in edges.items():
        x[:, :, j, c] = 0.02
    for v in range(2):
        for i in range(2):
            _, ring = oracle.detect(x[v, i], g.parity[v], g.eps)
            assert np.nonzero(ring)[0].tolist() == sorted(edges)
    y = apply(torch_cuda, g, x, prec)
    assert field_errors(y, oracle_of(g, x)).max() <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_full_state_256x128x256_sampled(torch_cuda, prec):
    """The 28-field hybrid mix on 256 x 128 x 256 (CTA pairs) at full size, sampled shells of every
    hybrid field inside, across and outside the star, and of other classes."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    g = W.grid_28_hybrid(256, 128, 256)
    x = W.star_state(g, seed=11)
    plan = Plan.from_grid(g, precision=prec)
    y = plan.apply(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    shells = [(v, i) for v in (14, 17, 24, 25) for i in (6, 30, 80, 140)] + [(0, 100), (20, 7)]
    ref = oracle.filter_shells(x, shells, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor, eps=g.eps)
    fmax = {v: max(np.abs(ref[n]).max() for n, s in enumerate(shells) if s[0] == v) for v, _ in shells}
    err = np.array([np.abs(y[v, i].cpu().numpy() - ref[n]).max() / fmax[v] for n, (v, i) in enumerate(shells)])
    assert err.max() <= TOL, shells[int(err.argmax())]


@pytest.mark.parametrize("prec", PRECS)
def test_tiny_scales_subnormals_and_eps(torch_cuda, prec):
    """Fields scaled to 1e-305 (subnormal values next to normal ones), to 1e+300, and eps comparable
    to the field: the screen's scale and its flagged inputs must not change any decision."""
    g = W.grid_28_hybrid(3, 16, 32)
    g.r = np.array([2.5, 9.5, 20.5])
    x = W.star_state(g, seed=21)
    hyb = [v for v in range(g.nvars) if g.kind[v] == HYB]
    x[hyb[0]] *= 1e-305
    x[hyb[1]] *= 1e300
    x[hyb[2]] *= 1e-11  # the atmosphere (1e-21) is now far below eps = 1e-12, the star above it
    y = apply(torch_cuda, g, x, prec)
    assert field_errors(y, oracle_of(g, x)).max() <= TOL
    g.eps = 1e-9
    y = apply(torch_cuda, g, x, prec)
    assert field_errors(y, oracle_of(g, x)).max() <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_full_state_128x64x128_sampled(torch_cuda, prec):
    """The 28-field hybrid workload at full size, in the launch configuration the benchmark times;
    the oracle checks sampled shells of every hybrid field (inside, across and outside the star)
    and of the other classes."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan
    wl = W.hybrid_state_128x64x128()
    g = wl.grids[0]
    x = wl.state()
    plan = Plan.from_grid(g, precision=prec)
    y = plan.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    shells = [(v, i) for v in (14, 15, 16, 17, 24, 25) for i in (3, 12, 25, 40, 64, 90)]
    shells += [(v, i) for v in (0, 18, 20, 26) for i in (5, 40, 127)]
    ref = oracle.filter_shells(x, shells, g.parity, g.kind, g.L, g.r, g.dr_min, g.floor, eps=g.eps)
    fmax = {v: max(np.abs(ref[n]).max() for n, s in enumerate(shells) if s[0] == v) for v, _ in shells}
    err = np.array([np.abs(y[v, i] - ref[n]).max() / fmax[v] for n, (v, i) in enumerate(shells)])
    assert err.max() <= TOL, shells[int(err.argmax())]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("Nr,Nth,Nph", [(4, 32, 64), (2, 128, 256)])
def test_in_place_fp32_host_and_batch(torch_cuda, prec, Nr, Nth, Nph):
    """In place (every row is moved: the choices depend on the data), FP32 storage (the detector
    sees the widened FP32 values), the host-buffer entry point and a CUDA-graph batch; one CTA and
    a CTA pair per shell."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Batch, Plan
    g, x = star_case(Nr, Nth, Nph, seed=31)
    ref = oracle_of(g, x)
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(x).cuda()
    plan.apply(xd, out=xd)
    torch.cuda.synchronize()
    assert field_errors(xd.cpu().numpy(), ref).max() <= TOL
    xf = x.astype(np.float32)
    yf = plan.apply(torch.from_numpy(xf).cuda()).cpu().numpy()
    assert field_errors(yf.astype(np.float64), oracle_of(g, xf.astype(np.float64))).max() <= 2e-6
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    plan.apply_host(xh, oh)
    torch.cuda.synchronize()
    assert field_errors(oh.numpy(), ref).max() <= TOL
    b = Batch([plan])
    xs, outs = [torch.from_numpy(x).cuda()], [torch.empty(g.shape, dtype=torch.float64, device="cuda")]
    b.capture(xs, outs, 2)
    b.launch()
    torch.cuda.synchronize()
    assert torch.equal(outs[0], plan.apply(plan.apply(xs[0])))
    assert plan.sync_status() == 0


def test_unsupported_calls(torch_cuda):
    """The switch is nonlinear: no adjoint and no fused tanh steps; no tensor-core form and no
    chunked FP64 kernel (lengths with prime factors above 3)."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan, SphFilterError
    g = W.grid_28_hybrid(2, 8, 16)
    plan = Plan.from_grid(g, precision=2)
    z = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    for call in (lambda: plan.apply_adjoint(z), lambda: plan.apply_tanh(z), lambda: plan.apply_adjoint_tanh(z, z)):
        with pytest.raises(SphFilterError):
            call()
    with pytest.raises(SphFilterError):
        Plan.from_grid(g, precision=1)
    with pytest.raises(SphFilterError):  # Nphi = 2 x 37: the chunked FP64 kernel has no detector
        Plan.from_grid(W.grid_28_hybrid(2, 8, 74), precision=0)
    # a plan without hybrid fields keeps its adjoint
    g2 = W.grid_28(2, 8, 16)
    Plan.from_grid(g2, precision=2).apply_adjoint(z)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", PRECS)
def test_autotune_and_allocation_free_call(torch_cuda, prec):
    """The autotuner times other launch shapes (512 threads, where the detector's walk runs four
    bands of rows; other FFT batch sizes): the filtered state does not depend on the shape, bit for
    bit. The allocation-free host call gives the device call's result."""
    torch = torch_cuda
    from paper_2305_01537_gb300 import Plan, binding
    g, x = star_case(3, 64, 128, seed=51)  # 688,128 points: within the allocation-free capacity
    plan = Plan.from_grid(g, precision=prec)
    xd = torch.from_numpy(x).cuda()
    want = plan.apply(xd)
    torch.cuda.synchronize()
    assert field_errors(want.cpu().numpy(), oracle_of(g, x)).max() <= TOL
    plan.autotune(xd, torch.empty_like(xd))
    assert torch.equal(plan.apply(xd), want)
    lib = binding.load()
    xh = torch.from_numpy(x).pin_memory()
    got = torch.empty_like(xh).pin_memory()
    st = lib.sph_filter_apply_host_noalloc(plan._h, xh.data_ptr(), got.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert np.array_equal(got.numpy(), want.cpu().numpy())
    assert plan.sync_status() == 0
