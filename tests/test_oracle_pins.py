"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle (oracle/sph_oracle.c) against something other than itself: values the
paper states, closed-form eigen-responses, the paper's own pole example, invariants, brute force
through an independently built dense operator, and an extended-precision build of the same source.
Paper references are to arXiv:2305.01537, Sec. II.C "Filtering algorithms".
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def nrm_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------- values the paper states

def test_filter_values_golden():
    rows = _rows("filter_values.txt")
    assert len(rows) >= 10
    for row in rows:
        kind, l, lmax, expected = int(row[0]), float(row[1]), float(row[2]), float(row[3])
        got = oracle.filter_value(kind, l, lmax)
        assert got == pytest.approx(expected, rel=1e-15, abs=1e-300), row


def test_cutoffs_golden():
    for row in _rows("cutoffs.txt"):
        r, dr, L, j, Nth, lm, mm = (float(row[0]), float(row[1]), float(row[2]), int(row[3]),
                                    int(row[4]), float(row[5]), float(row[6]))
        assert oracle.lmax(r, dr, L) == pytest.approx(lm, rel=1e-15)
        assert oracle.mmax(r, dr, L, j, Nth) == pytest.approx(mm, rel=1e-14)


def test_extended_precision_build_agrees_on_values():
    for kind in (0, 1, 2):
        for l in (0.0, 1.0, 5.0, 17.0, 63.0):
            a = oracle.filter_value(kind, l, 7.25)
            b = oracle.filter_value(kind, l, 7.25, variant="ld")
            assert a == pytest.approx(b, rel=4e-15, abs=1e-300)  # a few ulps of libm


# ---------------------------------------------------------------- brute force: dense operator

def _circulant_column(M, mult):
    """c[d] = (1/M) sum over the signed frequencies l in (-M/2, M/2] of mult(|l|) cos(2 pi l d / M):
    the real-space kernel of a convolution with an even real multiplier."""
    ls = np.arange(-((M - 1) // 2), M // 2 + 1)
    d = np.arange(M)
    return (np.array([mult(abs(l)) for l in ls])[None, :] *
            np.cos(2 * np.pi * np.outer(d, ls) / M)).sum(axis=1) / M


def _f(kind, l, lm):
    if kind == 0:
        return 1.0 if l <= lm else math.exp(-(l - lm))
    if kind == 1:
        return math.exp(math.log(0.9) * (l / (lm + 1)) ** 2)
    return 1.0 if l <= lm else 0.0


def _dense_filter(Nth, Nph, a, kind, r, L, dr=1.0, floor=2.0):
    """Dense matrix of the double filter on one shell built in real space from circulant kernels:
    theta pass = G^T C G with G the signed doubling permutation, then phi pass = block-diagonal ring
    circulants. Independent of the oracle's DFT code."""
    n = Nth * Nph
    M = 2 * Nth
    lm = max(floor, 2 * r / dr * L)
    c = _circulant_column(M, lambda l: _f(kind, l, lm))
    T = np.zeros((n, n))
    s = -1.0 if a else 1.0
    for k in range(Nph // 2):
        # circle position q -> (flat index, sign)
        pos = [(q * Nph + k, 1.0) if q < Nth else ((M - 1 - q) * Nph + k + Nph // 2, s) for q in range(M)]
        for q in range(M):
            iq, sq = pos[q]
            for qq in range(M):
                iqq, sqq = pos[qq]
                T[iq, iqq] += sq * sqq * c[(q - qq) % M]
    P = np.zeros((n, n))
    for j in range(Nth):
        th = (j + 0.5) * math.pi / Nth
        mm = max(floor, 2 * r / dr * math.sin(th) * L)
        cj = _circulant_column(Nph, lambda m: _f(kind, m, mm))
        for k in range(Nph):
            for kk in range(Nph):
                P[j * Nph + k, j * Nph + kk] = cj[(k - kk) % Nph]
    return P @ T, T, P


@pytest.mark.parametrize("Nth,Nph", [(1, 2), (2, 4), (3, 6), (4, 8), (6, 12), (8, 8), (5, 10)])
@pytest.mark.parametrize("a", [0, 1])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_brute_force_dense_operator(Nth, Nph, a, kind):
    r, L = 0.35 + 0.1 * Nth, 1.7
    F, T, P = _dense_filter(Nth, Nph, a, kind, r, L)
    x = np.random.default_rng(Nth * 100 + Nph + 7 * a + kind).standard_normal((1, 1, Nth, Nph))
    y = oracle.filter(x, [a], [kind], [L], [r])
    assert nrm_err(y.ravel(), F @ x.ravel()) < 1e-13
    yt = oracle.theta_pass(x, [a], [kind], [L], [r])
    assert nrm_err(yt.ravel(), T @ x.ravel()) < 1e-13
    yp = oracle.phi_pass(x, [a], [kind], [L], [r])
    assert nrm_err(yp.ravel(), P @ x.ravel()) < 1e-13
    # transpose (c-11): explicit dense transpose vs the oracle's F^T
    z = oracle.filter_T(x, [a], [kind], [L], [r])
    assert nrm_err(z.ravel(), F.T @ x.ravel()) < 1e-13


def test_extended_precision_bounds_oracle_rounding():
    wl = W.full_state_128x64x128()
    g = wl.grids[0]
    x = wl.state()[:, :3]  # 28 fields x 3 shells, all kinds and both parities
    y = oracle.filter(x, g.parity, g.kind, g.L, g.r[:3])
    y_ld = oracle.filter(x, g.parity, g.kind, g.L, g.r[:3], variant="ld")
    for v in range(x.shape[0]):
        assert nrm_err(y[v], y_ld[v]) < 2e-15


# ---------------------------------------------------------------- closed-form eigen-responses

def _mode(Nth, Nph, a, m, l, phase):
    th = W.theta_points(Nth)[:, None]
    ph = W.phi_points(Nph)[None, :]
    prof = np.cos(l * th) if (a + m) % 2 == 0 else np.sin(l * th)
    return prof * (np.cos(m * ph) if phase == 0 else np.sin(m * ph))


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("a", [0, 1])
def test_eigen_response(kind, a):
    """x = cos/sin(m phi) P_l(theta) is an eigenfunction of each ring and circle filter, so the output is
    f(l, l_max) f(m, m_max(theta_j)) x exactly (theta pass first, then the phi pass)."""
    Nth, Nph = 12, 24
    rng = np.random.default_rng(11 + kind + 3 * a)
    for r in (0.5, 1.5, 2.5):
        L = 1.0
        lm = max(2.0, 2 * r * L)
        for _ in range(6):
            m = int(rng.integers(0, Nph // 2))
            l = int(rng.integers(1 if (a + m) % 2 else 0, Nth))
            phase = int(rng.integers(0, 2)) if m > 0 else 0
            x = _mode(Nth, Nph, a, m, l, phase)
            th = W.theta_points(Nth)
            fm = np.array([_f(kind, m, max(2.0, 2 * r * math.sin(t) * L)) for t in th])
            expect = _f(kind, l, lm) * fm[:, None] * x
            y = oracle.filter(x[None, None], [a], [kind], [L], [r])[0, 0]
            assert np.abs(y - expect).max() < 2e-14, (r, m, l, phase)


def test_pass_order_is_theta_then_phi():
    """With an eigenfunction input, theta-then-phi gives the closed form; phi-then-theta does not,
    because after the phi pass the profile is no longer a single l mode (m_max varies with theta)."""
    Nth, Nph, a, kind, r, L = 16, 32, 0, 0, 0.5, 3.0
    x = _mode(Nth, Nph, a, 6, 8, 0)
    th = W.theta_points(Nth)
    fm = np.array([_f(kind, 6, max(2.0, 2 * r * math.sin(t) * L)) for t in th])
    expect = _f(kind, 8, max(2.0, 2 * r * L)) * fm[:, None] * x
    y = oracle.filter(x[None, None], [a], [kind], [L], [r])[0, 0]
    z = oracle.filter_T(x[None, None], [a], [kind], [L], [r])[0, 0]
    assert np.abs(y - expect).max() < 1e-14
    assert np.abs(z - expect).max() > 1e-3


# ---------------------------------------------------------------- band-limited inputs pass unchanged

@pytest.mark.parametrize("kind", [0, 2])
@pytest.mark.parametrize("a", [0, 1])
def test_low_modes_pass_unchanged(kind, a):
    """Because of the floor 2 in l_max and m_max, every mode with l <= 2 and m <= 2 passes the
    exponential and the sharp filters unchanged at every radius, the origin included."""
    Nth, Nph = 10, 16
    rng = np.random.default_rng(5 + a)
    x = np.zeros((1, 4, Nth, Nph))
    for i in range(4):
        for m in range(3):
            for l in range(3):
                for phase in (0, 1):
                    if (a + m) % 2 and l == 0:
                        continue
                    x[0, i] += rng.standard_normal() * _mode(Nth, Nph, a, m, l, phase)
    r = np.array([0.0, 0.2, 1.0, 9.0])
    y = oracle.filter(x, [a], [kind], [3.0], r)
    assert nrm_err(y, x) < 1e-14


def _frame(th, ph):
    """Orthonormal spherical frame (e_r, e_theta, e_phi) in Cartesian components."""
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    z = np.zeros_like(th * ph)
    er = np.stack([st * cp + z, st * sp + z, ct + z])
    et = np.stack([ct * cp + z, ct * sp + z, -st + z])
    ep = np.stack([-sp + z, cp + z, z])
    return er, et, ep


def test_pole_example_constant_cartesian_metric():
    """The paper's pole argument (Sec. II.C): a constant Cartesian metric projected on the spherical
    orthonormal frame has only |l|, |m| <= 2 content, so the exponential and sharp filters must return
    its components unchanged at every radius. The test also checks the paper's printed closed forms
    of gamma_rr, gamma_phiphi and gamma_thetaphi against the frame projection, and that the
    parity each component gets matters (odd components filtered as even ones are changed)."""
    rng = np.random.default_rng(2305)
    a, b, c, d, e, f = rng.standard_normal(6)
    G = np.array([[1 + a, b, c], [b, 1 + d, e], [c, e, 1 + f]])
    Nth, Nph = 16, 32
    th = W.theta_points(Nth)[:, None]
    ph = W.phi_points(Nph)[None, :]
    er, et, ep = _frame(th, ph)
    comp = lambda u, v: np.einsum("i...,ij,j...->...", u, G, v)
    g_rr, g_tt, g_pp = comp(er, er), comp(et, et), comp(ep, ep)
    g_rt, g_rp, g_tp = comp(er, et), comp(er, ep), comp(et, ep)
    # the paper's closed forms
    s, co = np.sin, np.cos
    paper_rr = ((a + 1) * s(th) ** 2 * co(ph) ** 2
                + s(ph) * (s(th) ** 2 * (2 * b * co(ph) + (d + 1) * s(ph)) + e * s(2 * th))
                + c * s(2 * th) * co(ph) + (f + 1) * co(th) ** 2)
    paper_pp = 0.5 * (2 + a + d + (-a + d) * co(2 * ph) - 2 * b * s(2 * ph))
    paper_tp = co(th) * ((d - a) * s(ph) * co(ph) + b * co(2 * ph)) + s(th) * (c * s(ph) - e * co(ph))
    assert np.abs(paper_rr - g_rr).max() < 1e-13
    assert np.abs(paper_pp - g_pp).max() < 1e-13
    assert np.abs(paper_tp - g_tp).max() < 1e-13
    fields = [g_rr, g_tt, g_pp, g_tp, g_rt, g_rp]
    parity = [0, 0, 0, 0, 1, 1]
    x = np.stack([np.broadcast_to(fl, (3, Nth, Nph)) for fl in fields])  # 3 shells each
    r = np.array([0.0, 0.5, 4.0])
    for kind in (0, 2):
        y = oracle.filter(x, parity, [kind] * 6, [3.0] * 6, r)
        for v in range(6):
            assert nrm_err(y[v], x[v]) < 1e-14, (kind, v)
    # wrong parity for the odd components breaks the smooth continuation over the pole
    y = oracle.filter(x[4:], [0, 0], [0, 0], [3.0, 3.0], r)
    assert nrm_err(y[0], x[4]) > 1e-3
    # the Gaussian filter damps even these low modes
    y = oracle.filter(x[2:3], [0], [1], [3.0], r)
    assert nrm_err(y[0], x[2]) > 1e-3


# ---------------------------------------------------------------- invariants

def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("a", [0, 1])
def test_sharp_filter_each_pass_idempotent(a):
    x = _rand((1, 3, 12, 24), 3 + a)
    r = np.array([0.5, 1.5, 2.5])
    for pas in (oracle.theta_pass, oracle.phi_pass):
        y = pas(x, [a], [2], [1.0], r)
        yy = pas(y, [a], [2], [1.0], r)
        assert nrm_err(yy, y) < 1e-14
        assert nrm_err(y, x) > 1e-3  # it is not the identity
    # composite: idempotent when the phi cutoff does not depend on theta (m_max >= Nphi/2 everywhere)
    r = np.array([40.0])
    y = oracle.filter(x[:, :1], [a], [2], [0.4], r)
    yy = oracle.filter(y, [a], [2], [0.4], r)
    assert nrm_err(yy, y) < 1e-14


def test_mean_preservation():
    x = _rand((2, 3, 10, 20), 9)
    r = np.array([0.5, 2.5, 7.5])
    for kind in (0, 1, 2):
        # phi pass keeps every ring mean (f(0) = 1)
        y = oracle.phi_pass(x, [0, 1], [kind] * 2, [1.0] * 2, r)
        assert np.abs(y.mean(axis=3) - x.mean(axis=3)).max() < 1e-14
        # the composite keeps the unweighted shell sum of an even field
        y = oracle.filter(x[:1], [0], [kind], [1.0], r)
        assert np.abs(y.sum(axis=(2, 3)) - x[:1].sum(axis=(2, 3))).max() < 1e-12
    # ... but not of an odd one: its circle mean mixes +x and -x
    y = oracle.filter(x[1:], [1], [0], [1.0], r)
    assert np.abs(y.sum(axis=(2, 3)) - x[1:].sum(axis=(2, 3))).max() > 1e-3


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_parseval_per_pass(kind):
    """||x||^2 - ||Tx||^2 = (1/N) sum_l (1 - f_l^2) |x_hat_l|^2, per ring (phi pass) and per doubled
    circle (theta pass); also ||Fx|| <= ||x||."""
    Nth, Nph, r, L, a = 8, 16, 1.5, 1.0, 1
    x = _rand((1, 1, Nth, Nph), 21 + kind)
    # phi pass
    y = oracle.phi_pass(x, [a], [kind], [L], [r])[0, 0]
    for j in range(Nth):
        mm = max(2.0, 2 * r * math.sin((j + 0.5) * math.pi / Nth) * L)
        X = np.fft.fft(x[0, 0, j])
        fl = np.array([_f(kind, abs(m if m <= Nph // 2 else m - Nph), mm) for m in range(Nph)])
        lhs = (x[0, 0, j] ** 2).sum() - (y[j] ** 2).sum()
        rhs = ((1 - fl ** 2) * np.abs(X) ** 2).sum() / Nph
        assert abs(lhs - rhs) < 1e-12 * (x[0, 0, j] ** 2).sum()
    # theta pass: per doubled circle
    y = oracle.theta_pass(x, [a], [kind], [L], [r])[0, 0]
    lm = max(2.0, 2 * r * L)
    M = 2 * Nth
    s = -1.0 if a else 1.0
    for k in range(Nph // 2):
        cin = np.concatenate([x[0, 0, :, k], s * x[0, 0, ::-1, k + Nph // 2]])
        cout = np.concatenate([y[:, k], s * y[::-1, k + Nph // 2]])
        X = np.fft.fft(cin)
        fl = np.array([_f(kind, abs(l if l <= M // 2 else l - M), lm) for l in range(M)])
        lhs = (cin ** 2).sum() - (cout ** 2).sum()
        rhs = ((1 - fl ** 2) * np.abs(X) ** 2).sum() / M
        assert abs(lhs - rhs) < 1e-12 * (cin ** 2).sum()
    y = oracle.filter(x, [a], [kind], [L], [r])
    assert (y ** 2).sum() <= (x ** 2).sum() * (1 + 1e-14)


@pytest.mark.parametrize("a", [0, 1])
def test_symmetries(a):
    """F commutes with phi shifts (the shift by Nphi/2 is the half-work pairing of the double
    covering), with the reflection phi -> -phi and with the equatorial reflection theta -> pi - theta."""
    Nth, Nph = 9, 16
    x = _rand((1, 2, Nth, Nph), 31 + a)
    r = np.array([0.5, 1.7])
    args = ([a], [0], [1.3], r)
    y = oracle.filter(x, *args)
    for shift in (1, 3, Nph // 2):
        ys = oracle.filter(np.roll(x, shift, axis=3), *args)
        assert nrm_err(ys, np.roll(y, shift, axis=3)) < 1e-14
    refl = lambda z: np.roll(z[..., ::-1], 1, axis=3)  # k -> -k mod Nphi
    assert nrm_err(oracle.filter(refl(x), *args), refl(y)) < 1e-14
    eq = lambda z: z[:, :, ::-1, :]
    assert nrm_err(oracle.filter(eq(x), *args), eq(y)) < 1e-14


def test_adjoint_identity():
    wl = W.full_state_128x64x128()
    g = wl.grids[0]
    sel = [0, 14, 18, 20, 24, 26]  # one field of each class and parity
    x = _rand((len(sel), 4, 16, 32), 41)
    yv = _rand((len(sel), 4, 16, 32), 42)
    par = [g.parity[v] for v in sel]
    knd = [g.kind[v] for v in sel]
    Ls = [g.L[v] for v in sel]
    r = np.array([0.5, 1.5, 3.5, 9.5])
    Fx = oracle.filter(x, par, knd, Ls, r)
    FTy = oracle.filter_T(yv, par, knd, Ls, r)
    lhs, rhs = (Fx * yv).sum(), (x * FTy).sum()
    assert abs(lhs - rhs) < 1e-13 * np.sqrt((x ** 2).sum() * (yv ** 2).sum())


def test_rejects_bad_arguments():
    x = np.zeros((1, 1, 4, 6))
    with pytest.raises(ValueError):
        oracle.filter(np.zeros((1, 1, 4, 5)), [0], [0], [3.0], [0.5])  # odd Nphi
    with pytest.raises(ValueError):
        oracle.filter(x, [2], [0], [3.0], [0.5])  # parity not 0/1
    with pytest.raises(ValueError):
        oracle.filter(x, [0], [5], [3.0], [0.5])  # unknown kind
    with pytest.raises(ValueError):
        oracle.filter(x, [0], [0], [0.0], [0.5])  # L <= 0
    with pytest.raises(ValueError):
        oracle.filter(x, [0], [0], [3.0], [-1.0])  # r < 0
    with pytest.raises(ValueError):
        oracle.filter(x, [0], [0], [3.0], [0.5], dr_min=0.0)
