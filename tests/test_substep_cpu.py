"""The toy substep loop (paper_2305_01537_gb300.substep) on the CPU, with the oracle as the filter:
solid-body rotation about the x axis on one shell, SSP-RK3, the filter after every substep
(Sec. II.C). Without the filter the step is bounded by the rings next to the poles; with it, a step
several times larger stays stable."""
import math

import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import substep as S


def oracle_filter(Nth, Nph, kind):
    r = np.array([Nph / 4.0])  # m_max reaches the Nyquist mode at the equator
    return lambda u: oracle.filter(u[None, None], [0], [kind], [1.0], r, 1.0, 2.0)[0, 0]


def test_rhs_is_exact_for_a_rigid_rotation_invariant():
    """A field that depends only on x = sin(theta) cos(phi) is invariant under rotation about the x
    axis: the right-hand side vanishes up to the O(h^2) error of the centred differences."""
    Nth, Nph = 32, 64
    th = (np.arange(Nth) + 0.5) * math.pi / Nth
    ph = 2 * math.pi * np.arange(Nph) / Nph
    u = np.sin(th)[:, None] * np.cos(ph)[None, :]
    P = S.RotationAdvection(Nth, Nph)
    assert np.abs(P.rhs(u)).max() < 5e-3
    # a field u = z = cos(theta) changes as du/dt = -(omega x r) . grad z = -Omega y
    v = np.cos(th)[:, None] * np.ones((1, Nph))
    expect = -np.sin(th)[:, None] * np.sin(ph)[None, :]
    assert np.abs(P.rhs(v) - expect).max() < 5e-3


@pytest.mark.parametrize("kind", [0, 2])
def test_filter_lifts_the_axis_step_limit(kind):
    Nth, Nph = 16, 32
    P = S.RotationAdvection(Nth, Nph)
    th_lim, ax_lim = P.cfl_steps()
    u0 = S.blob(Nth, Nph)
    dt = 0.5 * th_lim  # about 5 times the axis limit
    assert dt > 4 * ax_lim
    steps = int(round(4 * math.pi / dt))  # two rotations
    _, peaks_f = S.run(u0, steps, dt, P, oracle_filter(Nth, Nph, kind))
    assert max(peaks_f) <= 1.0 + 1e-12 and min(peaks_f) > 0.3
    with np.errstate(all="ignore"):
        _, peaks_u = S.run(u0, steps, dt, P, None)
    assert not (max(peaks_u) < 1e3)  # blows up (or overflows to inf/nan)
    # without the filter the axis limit holds
    dt = 0.9 * ax_lim
    _, peaks = S.run(u0, int(round(2 * math.pi / dt)), dt, P, None)
    assert max(peaks) <= 1.0 + 1e-12
