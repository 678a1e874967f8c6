"""Pins of the constraint-map oracle (Sec. II.C, constraints det(gamma_bar) = det(gamma_hat) and
gamma_bar^{ij} A_bar_ij = 0 with their substitutions and the modified form near BHs).

Each pin is checked by other means than the oracle's formula: the constraints themselves in the
coordinate basis (with explicit scale factors R = (1, r, r sin theta)), the linearity of the
determinant in m_11, closed forms for scaled identities and diagonal metrics, and constructions of
already-constrained states from an eigen-decomposition.
"""
import numpy as np
import pytest

from oracle import constraints as C


def random_state(n, seed, hscale=0.2):
    rng = np.random.default_rng(seed)
    h = hscale * rng.standard_normal((6, n))
    A = rng.standard_normal((6, n))
    return h, A, rng


def sym(c):
    return C._to_matrix(c)


def test_standard_form_meets_both_constraints_in_the_coordinate_basis():
    h, A, rng = random_state(200, 1)
    alpha = np.ones(200)
    h2, A2 = C.enforce(h, A, alpha, np.zeros(200, bool))
    r = rng.uniform(0.5, 50.0, 200)
    th = rng.uniform(0.05, np.pi - 0.05, 200)
    R = np.stack([np.ones(200), r, r * np.sin(th)], axis=-1)            # [n, 3]
    RR = R[:, :, None] * R[:, None, :]
    g_bar = RR * (np.eye(3) + sym(h2))                                   # coordinate components
    a_bar = RR * sym(A2)
    g_hat_det = np.prod(R ** 2, axis=-1)
    assert np.allclose(np.linalg.det(g_bar) / g_hat_det, 1.0, rtol=0, atol=1e-13)
    tr = np.einsum("nab,nab->n", np.linalg.inv(g_bar), a_bar)
    assert np.abs(tr).max() <= 1e-13 * np.abs(A).max()


def test_idempotent():
    h, A, rng = random_state(100, 2)
    alpha = rng.uniform(0.0, 1.0, 100)
    flag = rng.uniform(size=100) < 0.5
    h1, A1 = C.enforce(h, A, alpha, flag)
    h2, A2 = C.enforce(h1, A1, alpha, flag)
    assert np.abs(h2 - h1).max() <= 1e-14 and np.abs(A2 - A1).max() <= 1e-14 * np.abs(A1).max()


@pytest.mark.parametrize("c", [0.5, 1.0, 1.7, 3.0])
def test_scaled_identity_closed_form(c):
    """m = c I: the metric becomes flat (h = 0) and A loses its plain trace: A - I tr(A)/3."""
    n = 20
    h = np.zeros((6, n))
    h[[0, 3, 5]] = c - 1.0
    _, A, _ = random_state(n, 3)
    h2, A2 = C.enforce(h, A, np.ones(n), np.zeros(n, bool))
    assert np.abs(h2).max() <= 4e-16 * c
    trace = A[0] + A[3] + A[5]
    expect = A.copy()
    expect[[0, 3, 5]] -= trace / 3.0
    assert np.abs(A2 - expect).max() <= 1e-15 * np.abs(A).max() * 4


def test_constrained_state_is_unchanged():
    """det(m) = 1 and A = m^(1/2) B m^(1/2) with B symmetric and traceless already satisfy both
    constraints (tr(m^-1 A) = tr(B) = 0)."""
    rng = np.random.default_rng(4)
    n = 50
    out_h, out_A = np.empty((6, n)), np.empty((6, n))
    for k in range(n):
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        lam = rng.uniform(0.6, 1.6, 3)
        lam[2] = 1.0 / (lam[0] * lam[1])
        m = (q * lam) @ q.T
        s = (q * np.sqrt(lam)) @ q.T
        b = rng.standard_normal((3, 3))
        b = b + b.T
        b -= np.eye(3) * np.trace(b) / 3.0
        a = s @ b @ s
        out_h[:, k] = C._from_matrix(m - np.eye(3))
        out_A[:, k] = C._from_matrix(a)
    h2, A2 = C.enforce(out_h, out_A, np.ones(n), np.zeros(n, bool))
    assert np.abs(h2 - out_h).max() <= 1e-14 and np.abs(A2 - out_A).max() <= 1e-14 * np.abs(out_A).max()


def test_modified_form_diagonal_closed_form():
    """Diagonal m near a BH: h_11 = 1/(m_22 m_33) - 1, everything else kept."""
    rng = np.random.default_rng(5)
    n = 30
    h = np.zeros((6, n))
    h[[0, 3, 5]] = rng.uniform(-0.4, 0.4, (3, n))
    A = rng.standard_normal((6, n))
    h2, A2 = C.enforce(h, A, np.full(n, 0.1), np.ones(n, bool))
    m22, m33 = 1.0 + h[3], 1.0 + h[5]
    assert np.abs(h2[0] - (1.0 / (m22 * m33) - 1.0)).max() <= 1e-15
    assert np.array_equal(h2[1:], h[1:]) and np.array_equal(A2, A)


def test_modified_form_solves_the_determinant_for_m11():
    """det(m) is linear in m_11: det = m_11 M + c. Evaluating it at m_11 = 0 and 1 (numpy's det)
    gives the m_11 with det = 1, which the modified form must reproduce."""
    h, A, rng = random_state(100, 6)
    h2, A2 = C.enforce(h, A, np.full(100, 0.05), np.ones(100, bool))
    m = sym(h) + np.eye(3)
    m0, m1 = m.copy(), m.copy()
    m0[:, 0, 0] = 0.0
    m1[:, 0, 0] = 1.0
    d0, d1 = np.linalg.det(m0), np.linalg.det(m1)
    m11 = (1.0 - d0) / (d1 - d0)
    assert np.abs(h2[0] - (m11 - 1.0)).max() <= 1e-13
    assert np.array_equal(h2[1:], h[1:]) and np.array_equal(A2, A)


def test_modified_form_matches_the_coordinate_basis_formula():
    """The paper's h_11 formula is written with coordinate components gamma_bar_ij, det(gamma_hat)
    and the scale factor R_1: evaluated that way it gives the oracle's orthonormal value."""
    h, A, rng = random_state(100, 7)
    h2, _ = C.enforce(h, A, np.zeros(100), np.ones(100, bool))
    r = rng.uniform(0.5, 50.0, 100)
    th = rng.uniform(0.05, np.pi - 0.05, 100)
    R = np.stack([np.ones(100), r, r * np.sin(th)], axis=-1)
    g = (R[:, :, None] * R[:, None, :]) * (np.eye(3) + sym(h))
    g_hat = np.prod(R ** 2, axis=-1)
    g12, g13, g22, g23, g33 = g[:, 0, 1], g[:, 0, 2], g[:, 1, 1], g[:, 1, 2], g[:, 2, 2]
    h11 = (g_hat + g12 ** 2 * g33 - 2 * g12 * g13 * g23 + g13 ** 2 * g22) / (g22 * g33 - g23 ** 2) / (R[:, 0] ** 2) - 1
    assert np.abs(h2[0] - h11).max() <= 1e-13


def test_branch_selection():
    """Modified form iff the theta filter is active and alpha < alpha_bh (strictly)."""
    h, A, _ = random_state(4, 8)
    alpha = np.array([0.3, np.nextafter(0.3, 0.0), 0.1, 0.1])
    flag = np.array([True, True, False, True])
    h2, A2 = C.enforce(h, A, alpha, flag)
    hs, As = C.enforce(h, A, alpha, np.zeros(4, bool))
    bh = np.array([False, True, False, True])
    assert np.array_equal(A2[:, bh], A[:, bh]) and np.array_equal(h2[1:, bh], h[1:, bh])
    assert np.array_equal(h2[:, ~bh], hs[:, ~bh]) and np.array_equal(A2[:, ~bh], As[:, ~bh])
    h3, A3 = C.enforce(h, A, alpha, flag, alpha_bh=0.05)  # no point below: all standard
    assert np.array_equal(h3, hs) and np.array_equal(A3, As)
