"""Pins of the oracle's hybrid filter (CPU only): arXiv:2305.01537, Sec. II.C, the switch between
the exponential and the Gaussian filter by Jameson's shock detector
    sigma_i = |u_{i-1} - 2 u_i + u_{i+1}| / (|u_{i-1}| + 2 |u_i| + |u_{i+1}| + eps),
with the Gaussian filter for a theta circle or phi ring in which some cell has sigma >= 0.95.

The detector is pinned by closed forms of sigma and by tiny shells worked out by hand (the double
covering's neighbours across the pole with the parity sign); the selection is pinned against the
exponential and Gaussian filters, which the other pin files fix on their own.
"""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

EXP, GAUSS, HYB = 0, 1, 3


# ---------------------------------------------------------------- closed forms of sigma

@pytest.mark.parametrize("x,fires", [(0.0, True), (0.01, True), (0.02, True), (0.025, True), (0.0256, True),
                                     (0.0257, False), (0.03, False), (0.5, False), (1.0, False)])
def test_sigma_of_a_dip(x, fires):
    """u = (1, x, 1), 0 <= x <= 1, eps = 0: sigma = (2 - 2x) / (2 + 2x) = (1 - x) / (1 + x), which
    reaches 0.95 at x = 1/39 = 0.025641..."""
    assert ((1 - x) / (1 + x) >= 0.95) == fires  # the closed form itself
    assert oracle.jameson_fires(1.0, x, 1.0, 0.0) == fires


@pytest.mark.parametrize("eps,fires", [(0.0, True), (1e-12, True), (1e-11, True), (2e-11, False), (1.0, False)])
def test_sigma_of_a_spike_and_eps(eps, fires):
    """u = (0, 1e-10, 0): sigma = 2e-10 / (2e-10 + eps): 1, 0.990, 0.952, 0.909, ~0."""
    assert oracle.jameson_fires(0.0, 1e-10, 0.0, eps) == fires


def test_sigma_special_sequences():
    assert oracle.jameson_fires(1.0, -1.0, 1.0, 0.0)        # alternating signs: sigma = 4/4
    assert oracle.jameson_fires(-3.0, 3.0, -3.0, 1e-12)
    assert oracle.jameson_fires(1.0, 0.0, 0.0, 1e-12)       # next to a step from 0: sigma = 1/(1+eps)
    assert not oracle.jameson_fires(0.0, 1.0, 1.0, 0.0)     # on the step: 1/3
    assert not oracle.jameson_fires(2.5, 2.5, 2.5, 0.0)     # constant: 0
    assert not oracle.jameson_fires(1.0, 2.0, 3.0, 0.0)     # linear: 0
    assert not oracle.jameson_fires(-1.0, 1.0, 1.0, 0.0)    # a sign flip between equal magnitudes: 1/2
    assert not oracle.jameson_fires(0.0, 0.0, 0.0, 1e-12)   # 0 / eps
    assert not oracle.jameson_fires(0.0, 0.0, 0.0, 0.0)     # 0 / 0 is not >= 0.95


def test_sigma_invariances():
    """sigma is symmetric in the two neighbours, odd-even in a common sign, and (eps = 0) invariant
    under scaling by powers of two (exact in binary floating point)."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a, b, c = rng.standard_normal(3) * 10.0 ** rng.integers(-5, 5, size=3)
        f = oracle.jameson_fires(a, b, c, 0.0)
        assert oracle.jameson_fires(c, b, a, 0.0) == f
        assert oracle.jameson_fires(-a, -b, -c, 0.0) == f
        assert oracle.jameson_fires(a * 2.0 ** 40, b * 2.0 ** 40, c * 2.0 ** 40, 0.0) == f
        assert oracle.jameson_fires(a * 2.0 ** -40, b * 2.0 ** -40, c * 2.0 ** -40, 0.0) == f


# ---------------------------------------------------------------- detector flags on tiny shells

def test_detect_hand_worked_2x4():
    """Ntheta = 2, Nphi = 4: circles k = 0 (meridians 0, 2) and k = 1 (meridians 1, 3), 4 samples each:
    circle k = (x[0][k], x[1][k], s x[1][k+2], s x[0][k+2]), s = (-1)^a.
        x = [[ 1, 1, 1, 1],
             [-1, 1,-1, 1]]
    Circle 0 is (1, -1, -1, 1) for a = 0 (every cell: a sign flip between equal magnitudes,
    sigma = 1/2) and (1, -1, 1, -1) for a = 1 (alternating: sigma = 1). Circle 1 is constant
    (a = 0) or (1, 1, -1, -1) (a = 1, sigma = 1/2). Ring 0 is constant, ring 1 alternates."""
    x = np.array([[1.0, 1.0, 1.0, 1.0], [-1.0, 1.0, -1.0, 1.0]])
    circ, ring = oracle.detect(x, 0, 1e-12)
    assert circ.tolist() == [False, False] and ring.tolist() == [False, True]
    circ, ring = oracle.detect(x, 1, 1e-12)
    assert circ.tolist() == [True, False] and ring.tolist() == [False, True]


def test_detect_hand_worked_spikes_3x6():
    """Ntheta = 3, Nphi = 6 (circles k = 0, 1, 2 join meridians k and k + 3).
    A single spike fires the ring and the circle that hold it: the spike cell (0, 1, 0) and its
    neighbours (1, 0, 0) have sigma ~ 1; all-zero rings and circles give 0 / eps."""
    x = np.zeros((3, 6))
    x[1, 4] = 1.0
    for a in (0, 1):
        circ, ring = oracle.detect(x, a, 1e-12)
        assert circ.tolist() == [False, True, False]
        assert ring.tolist() == [False, True, False]
    # a spike on the row next to the north pole, meridian 5: its circle (k = 2) also walks meridian
    # 2, across the pole; ring 0 holds it
    x = np.zeros((3, 6))
    x[0, 5] = 1.0
    circ, ring = oracle.detect(x, 1, 1e-12)
    assert circ.tolist() == [False, False, True] and ring.tolist() == [True, False, False]


def test_detect_across_the_pole_depends_on_parity():
    """Ntheta = 3, Nphi = 4. Meridian 0 = (0, 1, 2) and meridian 2 = (1, 2, 0) from the north pole
    down; meridians 1 and 3 are constant. Circle 0 = (x00, x10, x20, s x22, s x12, s x02):
      s = -1: (0, 1, 2, 0, -2, -1), a triangle wave: sigma = 0, 0, 3/5, 0, 3/5, 0 (quiet);
      s = +1: (0, 1, 2, 0, 2, 1): the pole cells q = 0 (neighbours 1, 1 around 0) and q = 3
              (2, 2 around 0) have sigma = 1 (fire).
    Rings: row 0 = (0, 5, 1, 5) and row 2 = (2, 5, 0, 5) hold a 0 between two 5s (fire); row 1 =
    (1, 5, 2, 5) peaks at sigma = 2/3."""
    x = np.array([[0.0, 5.0, 1.0, 5.0], [1.0, 5.0, 2.0, 5.0], [2.0, 5.0, 0.0, 5.0]])
    circ, ring = oracle.detect(x, 0, 1e-12)
    assert circ.tolist() == [True, False] and ring.tolist() == [True, False, True]
    circ, ring = oracle.detect(x, 1, 1e-12)
    assert circ.tolist() == [False, False] and ring.tolist() == [True, False, True]
    # a spike across the pole fires its circle for either sign: circle 0 = (0, 0, 0, 0, 0, s)
    x = np.zeros((3, 4))
    x[0, 2] = 1.0
    for a in (0, 1):
        assert oracle.detect(x, a, 1e-12)[0].tolist() == [True, False]


def test_detect_smooth_fields_are_quiet():
    """Smooth even fields (few low modes) offset away from zero never fire: sigma is then O(h^2)."""
    g = W.Grid(4, 32, 64, [0], [HYB], [3.0])
    x = W.few_mode_state(g, seed=3, nmodes=4, mode_max=3, noise=0.0) + 10.0
    for i in range(g.Nr):
        circ, ring = oracle.detect(x[0, i], 0, 1e-12)
        assert not circ.any() and not ring.any()


# ---------------------------------------------------------------- selection against exp / Gaussian

def _args(g):
    return g.parity, g.kind, g.L, g.r, g.dr_min, g.floor


def test_quiet_hybrid_is_the_exponential_filter():
    g = W.Grid(3, 16, 32, [0, 0], [HYB, EXP], [3.0, 3.0], r=np.array([0.5, 1.5, 2.5]))
    x = W.few_mode_state(g, seed=4, nmodes=5, mode_max=4, noise=0.0) + 5.0
    x[1] = x[0]
    y = oracle.filter(x, *_args(g), eps=1e-12)
    assert np.array_equal(y[0], y[1])


def test_rough_hybrid_is_the_gaussian_filter():
    """A checkerboard on top of a smooth field makes every ring and circle fire."""
    g = W.Grid(3, 16, 32, [0, 1], [HYB, HYB], [3.0, 3.0], r=np.array([0.5, 1.5, 2.5]))
    x = W.few_mode_state(g, seed=4, nmodes=5, mode_max=4, noise=0.0)
    x += 100.0 * (-1.0) ** np.add.outer(np.arange(16), np.arange(32))[None, None]
    y = oracle.filter(x, *_args(g), eps=1e-12)
    gg = W.Grid(3, 16, 32, [0, 1], [GAUSS, GAUSS], [3.0, 3.0], r=g.r)
    assert np.array_equal(y, oracle.filter(x, *_args(gg)))


def test_mixed_selection_per_ring_and_circle():
    """Spikes in a few rows and meridians: each pass alone equals the Gaussian pass on the circles
    or rings that hold a firing cell and the exponential pass elsewhere, value for value; the whole
    filter is the theta pass with the circles' choice followed by the phi pass with the rings'
    choice, both taken on the filter's input."""
    Nth, Nph = 12, 24
    g = W.Grid(2, Nth, Nph, [1], [HYB], [2.0], r=np.array([1.5, 3.5]))
    ge = W.Grid(2, Nth, Nph, [1], [EXP], [2.0], r=g.r)
    gg = W.Grid(2, Nth, Nph, [1], [GAUSS], [2.0], r=g.r)
    x = W.few_mode_state(g, seed=6, nmodes=4, mode_max=3, noise=0.0)
    x[0, :, 3, 5] += 50.0
    x[0, 1, 8, 19] += 50.0
    x[0, 1, 0, 2] -= 50.0
    flags = [oracle.detect(x[0, i], 1, g.eps) for i in range(2)]
    assert any(c.any() and not c.all() for c, _ in flags) and any(r.any() and not r.all() for _, r in flags)
    eps = g.eps
    th = oracle.theta_pass(x, *_args(g), eps=eps)
    th_e, th_g = oracle.theta_pass(x, *_args(ge)), oracle.theta_pass(x, *_args(gg))
    ph = oracle.phi_pass(x, *_args(g), eps=eps)
    ph_e, ph_g = oracle.phi_pass(x, *_args(ge)), oracle.phi_pass(x, *_args(gg))
    for i, (circ, ring) in enumerate(flags):
        cols = np.concatenate([circ, circ])  # circle k holds meridians k and k + Nphi/2
        assert np.array_equal(th[0, i][:, cols], th_g[0, i][:, cols])
        assert np.array_equal(th[0, i][:, ~cols], th_e[0, i][:, ~cols])
        assert np.array_equal(ph[0, i][ring], ph_g[0, i][ring])
        assert np.array_equal(ph[0, i][~ring], ph_e[0, i][~ring])
    # the full filter: detection on the input for both passes
    y = oracle.filter(x, *_args(g), eps=eps)
    t_e, t_g = oracle.phi_pass(th, *_args(ge)), oracle.phi_pass(th, *_args(gg))
    for i, (_, ring) in enumerate(flags):
        assert np.array_equal(y[0, i][ring], t_g[0, i][ring])
        assert np.array_equal(y[0, i][~ring], t_e[0, i][~ring])


def test_hybrid_extended_precision_build_agrees():
    g = W.grid_28_hybrid(3, 16, 32)
    g.r = np.array([2.5, 7.5, 12.5])
    x = W.star_state(g, seed=8)
    a = oracle.filter(x, *_args(g), eps=g.eps)
    b = oracle.filter(x, *_args(g), variant="ld", eps=g.eps)
    for v in range(g.nvars):
        assert np.abs(a[v] - b[v]).max() <= 1e-14 * max(np.abs(b[v]).max(), 1e-300)


def test_hybrid_rejects_transpose_and_bad_eps():
    g = W.Grid(1, 4, 8, [0], [HYB], [3.0])
    x = np.zeros(g.shape)
    with pytest.raises(ValueError):
        oracle.filter_T(x, *_args(g), eps=1e-12)
    with pytest.raises(ValueError):
        oracle.filter(x, *_args(g), eps=-1.0)
    with pytest.raises(ValueError):
        oracle.filter(x, g.parity, [4], g.L, g.r)
