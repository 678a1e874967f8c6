"""Oracle for the algebraic-constraint map applied after filtering (arXiv:2305.01537, Sec. II.C,
"Filtering spacetime fields in the presence of BHs": the constraints det(gamma_bar) = det(gamma_hat)
and gamma_bar^{ij} A_bar_ij = 0, the substitutions that enforce them, and the modified form used
where the theta filter is active and the lapse is below 0.3).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline leg
are the only callers allowed. It imports nothing from the product package.

Readings (the paper states the map in the notation of its SphericalNR references):
- The metric and curvature components are orthonormal-basis components h_{ab}, A_{ab}, with
  gamma_bar_ij = R_i R_j (delta_ij + h_ij) and gamma_hat_ij = diag(R_i^2) for the spherical
  background's scale factors R = (1, r, r sin theta). Hence det(gamma_hat)/det(gamma_bar) =
  1/det(m) with m = delta + h, and gamma_bar^{ij} A_bar_ij = sum_ab (m^-1)_ab A_ab: the scale
  factors cancel, and the map acts on m and A alone.
- Standard form: m -> det(m)^(-1/3) m (so det = 1), then A -> A - m tr/3 with tr = sum (m^-1)_ab
  A_ab; taking m and tr both before or both after the first substitution gives the same A.
- Modified form, where the caller flags that the theta filter is active and alpha < alpha_bh
  (strictly; 0.3 in the paper): h_11 is solved from det(gamma_bar) = det(gamma_hat) with the other
  components kept, the paper's closed form with the scale factors divided out; A is left as is.
- Components are ordered (11, 12, 13, 22, 23, 33).
"""
from __future__ import annotations

import numpy as np

ORDER = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def _to_matrix(c):
    """[6, ...] symmetric components -> [..., 3, 3]."""
    c = np.asarray(c, dtype=np.float64)
    out = np.empty(c.shape[1:] + (3, 3))
    for n, (a, b) in enumerate(ORDER):
        out[..., a, b] = c[n]
        out[..., b, a] = c[n]
    return out


def _from_matrix(m):
    return np.stack([m[..., a, b] for (a, b) in ORDER])


def enforce(h, A, alpha, theta_filtered, alpha_bh: float = 0.3):
    """The constraint map at every point.

    h, A: [6, ...] orthonormal components; alpha: [...] lapse; theta_filtered: [...] bool (True
    where the theta filter is active), broadcast against alpha. Returns (h', A')."""
    h = np.asarray(h, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    bh = np.broadcast_to(np.asarray(theta_filtered, dtype=bool), alpha.shape) & (alpha < alpha_bh)

    m = _to_matrix(h) + np.eye(3)
    a = _to_matrix(A)

    # standard form: det(m) -> 1, then the trace of A in the new metric removed
    det = np.linalg.det(m)
    m_std = m / np.cbrt(det)[..., None, None]
    tr = np.einsum("...ab,...ab->...", np.linalg.inv(m_std), a)
    a_std = a - m_std * (tr / 3.0)[..., None, None]

    # modified form: h_11 from det = 1 with the other components kept; A unchanged
    m12, m13, m22, m23, m33 = m[..., 0, 1], m[..., 0, 2], m[..., 1, 1], m[..., 1, 2], m[..., 2, 2]
    h11_bh = (1.0 + m12 * m12 * m33 - 2.0 * m12 * m13 * m23 + m13 * m13 * m22) / (m22 * m33 - m23 * m23) - 1.0

    h_out = _from_matrix(m_std - np.eye(3))
    a_out = _from_matrix(a_std)
    h_out[0] = np.where(bh, h11_bh, h_out[0])
    for n in range(1, 6):
        h_out[n] = np.where(bh, h[n], h_out[n])
    a_out = np.where(bh[None], A, a_out)
    return h_out, a_out
