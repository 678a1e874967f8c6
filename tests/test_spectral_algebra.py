"""The algebra behind the spectral form (SPH_PREC_SPECTRAL), checked on the CPU against the oracle.

The filter of Sec. II.C (theta pass on the doubled great circles, then phi pass on the rings) is
composed in azimuthal-mode space: with X_j the phi spectrum of ring j, shifting phi by pi multiplies
mode m by (-1)^m, so the doubled circle of mode m is X_q[m] (q < Ntheta) followed by
(-1)^(a + m) X_{2 Ntheta - 1 - q}[m], and F = Phi^-1 D T Phi. The GPU form evaluates T per mode
through a complex FFT of length Ntheta: v_n = z_2n, v_{N-1-n} = z_{2n+1} (z_j = X_j[m], times
(-1)^j for odd extensions), U_l = a_l V_l + b_l V_{N-l} with a_l = g_l + g_{N-l},
b_l = +-(g_l - g_{N-l}) e^{i pi l / N}, g_l = f(l) / (2 Ntheta), and the inverse steps. This file
restates those steps with numpy's FFT and checks them against the oracle's naive DFT filter, so
that a wrong sign, index or normalisation in the derivation fails here before any kernel runs.
"""
import numpy as np
import pytest

import oracle
from paper_2305_01537_gb300 import workloads as W


def theta_filter_mode(y, odd, g):
    """T for one mode: y the Ntheta values X_j[m], g the multipliers f(l)/(2 Ntheta), l = 0..Ntheta."""
    N = len(y)
    j = np.arange(N)
    sg = np.where(odd & (j % 2 == 1), -1.0, 1.0)
    z = sg * y
    v = np.empty(N, complex)
    v[: N // 2] = z[0::2]
    v[N // 2:] = z[1::2][::-1]
    V = np.fft.fft(v)
    l = np.arange(N)
    gl, gn = g[l], g[N - l]
    a = gl + gn
    b = (gn - gl if odd else gl - gn) * np.exp(1j * np.pi * l / N)
    U = a * V + b * V[(-l) % N]
    u = np.fft.fft(U.conj()).conj()  # unnormalised inverse
    w = np.empty(N, complex)
    w[0::2] = u[: N // 2]
    w[1::2] = u[N // 2:][::-1]
    return sg * w


def spectral_filter(x, g: W.Grid, transpose=False):
    out = np.empty_like(x)
    Nth, Nph = g.Ntheta, g.Nphi
    nh = Nph // 2 + 1
    for v in range(g.nvars):
        for i in range(g.Nr):
            lm = oracle.lmax(g.r[i], g.dr_min, g.L[v], g.floor)
            gth = np.array([oracle.filter_value(g.kind[v], l, lm) for l in range(Nth + 1)]) / (2 * Nth)
            D = np.array([[oracle.filter_value(g.kind[v], m, oracle.mmax(g.r[i], g.dr_min, g.L[v], jj, Nth, g.floor))
                           for m in range(nh)] for jj in range(Nth)])
            X = np.fft.rfft(x[v, i], axis=1)  # [Nth][nh]
            if transpose:
                X = X * D
            for m in range(nh):
                X[:, m] = theta_filter_mode(X[:, m], ((g.parity[v] + m) % 2) == 1, gth)
            if not transpose:
                X = X * D
            out[v, i] = np.fft.irfft(X, n=Nph, axis=1)
    return out


@pytest.mark.parametrize("Nth,Nph", [(2, 4), (4, 8), (6, 12), (8, 16), (16, 12), (12, 32)])
def test_spectral_composition_matches_the_oracle(Nth, Nph):
    parity = [0, 1, 0, 1, 0, 1]
    kind = [0, 0, 1, 1, 2, 2]
    L = [0.7, 1.3, 2.0, 0.5, 0.9, 1.1]
    r = np.array([0.0, 0.3, 1.1, 2.6, 7.0, 40.0])
    g = W.Grid(len(r), Nth, Nph, parity, kind, L, r)
    x = W.random_state(g.shape, seed=Nth * 100 + Nph)
    args = (g.parity, g.kind, g.L, g.r, g.dr_min, g.floor)
    ref = oracle.filter(x, *args)
    y = spectral_filter(x, g)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    reft = oracle.filter_T(x, *args)
    yt = spectral_filter(x, g, transpose=True)
    assert np.abs(yt - reft).max() <= 1e-13 * np.abs(reft).max()


def test_one_mode_against_the_doubled_circle():
    """T for one mode equals the filter of the (anti)symmetric doubled circle, computed directly."""
    rng = np.random.default_rng(4)
    for N in (2, 4, 6, 8, 16, 24):
        g = rng.uniform(0.0, 1.0, N + 1) / (2 * N)
        for odd in (False, True):
            y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
            c = np.concatenate([y, (-1.0 if odd else 1.0) * y[::-1]])
            l = np.arange(2 * N)
            direct = np.fft.ifft(np.fft.fft(c) * g[np.minimum(l, 2 * N - l)] * (2 * N))[:N]
            assert np.abs(theta_filter_mode(y, odd, g) - direct).max() <= 1e-14
