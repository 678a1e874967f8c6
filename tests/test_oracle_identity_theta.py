"""Pins of the fact the split launch rests on (Sec. II.C filters, exponential and sharp kinds).

The theta circles have 2 Ntheta points, so their highest mode is l = Ntheta. The exponential and the
sharp filter are exactly 1 for l <= l_max. So when l_max >= Ntheta the theta pass is the identity,
and the filter acts ring by ring: each ring is filtered on its own in phi. Just below the threshold
(l_max = Ntheta - 1/2) the top mode is damped, and the theta pass is no longer the identity.

The ring-by-ring reference is independent of the oracle: numpy's real FFT of each ring, times
f(m, m_max(r, theta_j)) from the oracle's filter values (pinned to the paper's formulas elsewhere),
then the inverse FFT.
"""
import numpy as np
import pytest

import oracle

EXP, SHARP = oracle.KIND_EXP, oracle.KIND_SHARP


def ring_by_ring(x, kind, L, r, dr_min=1.0, floor=2.0):
    """[nvars=1][Nr][Ntheta][Nphi] filtered ring by ring in phi (numpy FFT)."""
    _, Nr, Nth, Nph = x.shape
    y = np.empty_like(x)
    m = np.arange(Nph // 2 + 1)
    for i in range(Nr):
        for j in range(Nth):
            mm = oracle.mmax(r[i], dr_min, L, j, Nth, floor)
            f = np.array([oracle.filter_value(kind, float(k), mm) for k in m])
            y[0, i, j] = np.fft.irfft(np.fft.rfft(x[0, i, j]) * f, n=Nph)
    return y


def nrm(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("kind", [EXP, SHARP])
@pytest.mark.parametrize("Nth,Nph", [(8, 16), (9, 24), (16, 32)])
@pytest.mark.parametrize("parity", [0, 1])
def test_identity_theta_pass_at_and_above_threshold(kind, Nth, Nph, parity):
    L = 1.5
    r = np.array([Nth / (2 * L), Nth / (2 * L) + 0.7, 3.0 * Nth])  # l_max = Ntheta exactly, above, far above
    for ri in r:
        assert oracle.lmax(ri, 1.0, L) >= Nth
    rng = np.random.default_rng(Nth * 10 + parity + 100 * kind)
    x = rng.standard_normal((1, len(r), Nth, Nph))
    args = ([parity], [kind], [L], r)
    assert nrm(oracle.theta_pass(x, *args), x) <= 1e-14
    assert nrm(oracle.filter(x, *args), ring_by_ring(x, kind, L, r)) <= 1e-13


@pytest.mark.parametrize("kind", [EXP, SHARP])
@pytest.mark.parametrize("Nth,Nph", [(8, 16), (16, 32)])
def test_theta_pass_acts_just_below_threshold(kind, Nth, Nph):
    L = 1.5
    r = np.array([(Nth - 0.5) / (2 * L)])  # l_max = Ntheta - 1/2: the top mode l = Ntheta is damped
    assert oracle.lmax(r[0], 1.0, L) < Nth
    rng = np.random.default_rng(7 + Nth + kind)
    x = rng.standard_normal((1, 1, Nth, Nph))
    y = oracle.theta_pass(x, [0], [kind], [L], r)
    assert nrm(y, x) > 1e-3


def test_filter_commutes_with_per_ring_scales_above_threshold():
    """F(D x) = D F(x) for a per-ring diagonal D when the theta pass is the identity, against the
    ring-by-ring reference, within the oracle's field-relative accuracy. (Relative to a small
    ring's own size the oracle is less accurate: its theta round trip with unit multipliers carries
    rounding of the large rings into the small ones.)"""
    Nth, Nph, L = 16, 32, 4.0
    r = np.array([5.0, 8.0, 12.0])
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, len(r), Nth, Nph))
    d = np.ldexp(1.0, (np.arange(Nth) % 5) * 10 - 20)[None, None, :, None]
    ref = ring_by_ring(x, EXP, L, r) * d
    assert nrm(oracle.filter(x * d, [0], [EXP], [L], r), ref) <= 1e-13
