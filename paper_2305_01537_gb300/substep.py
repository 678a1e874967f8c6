"""Toy substep loop: the filter inside a Runge-Kutta integrator (Sec. II.C: the filter is applied to
every evolved field after each substep, so that the modes that would violate the CFL condition
near the polar axis never grow).

The equation is the advection of a scalar u(theta, phi) on one spherical shell by a solid-body
rotation with angular velocity Omega about the x axis. In spherical components the velocity is
v_theta = -Omega R sin(phi), v_phi = -Omega R cos(theta) cos(phi), so

    du/dt = Omega sin(phi) du/dtheta + Omega cot(theta) cos(phi) du/dphi.

The azimuthal speed grows like cot(theta) near the axis: with centred differences the explicit
step is limited by the rings next to the poles, about (sqrt(3) / Omega) dphi tan(theta_0) for
SSP-RK3, far below the theta limit sqrt(3) dtheta / Omega. The filter keeps only azimuthal modes
m <= m_max(theta) ~ sin(theta), which lifts that limit to roughly the equatorial one.

Derivatives are second-order centred differences on the double covering of Sec. II.C (the theta
stencil crosses the pole onto meridian phi + pi with the field's parity sign; u is a scalar, so
even) and periodic in phi. The time integrator is the three-stage strong-stability-preserving
Runge-Kutta method of Shu and Osher. The filter is any callable mapping a [Ntheta, Nphi] tensor to
its filtered copy; `plan_filter` builds one from a plan of this package (the CUDA kernels).
"""
from __future__ import annotations

import math
from typing import Callable

import numpy as np

Filter = Callable[["object"], "object"]


class RotationAdvection:
    """Right-hand side of the rotation problem on an Ntheta x Nphi cell-centred grid."""

    def __init__(self, Ntheta: int, Nphi: int, omega: float = 1.0, xp=np, device=None):
        """xp: numpy, or torch (the coefficients then live on `device`)."""
        if Nphi % 2:
            raise ValueError("Nphi must be even (the theta stencil crosses onto phi + pi)")
        self.Nth, self.Nph, self.omega, self.xp, self.device = Ntheta, Nphi, omega, xp, device
        th = (np.arange(Ntheta) + 0.5) * math.pi / Ntheta
        ph = 2 * math.pi * np.arange(Nphi) / Nphi
        self.dth, self.dph = math.pi / Ntheta, 2 * math.pi / Nphi
        a = omega * np.sin(ph)[None, :] * np.ones((Ntheta, 1))               # coefficient of du/dtheta
        b = omega * (np.cos(th) / np.sin(th))[:, None] * np.cos(ph)[None, :]  # coefficient of du/dphi
        self.a, self.b = self._to(a), self._to(b)

    def _to(self, arr):
        if self.xp is np:
            return arr
        return self.xp.as_tensor(arr, device=self.device)

    def _roll(self, u, shift, axis):
        if self.xp is np:
            return np.roll(u, shift, axis=axis)
        return self.xp.roll(u, shifts=shift, dims=axis)

    def rhs(self, u):
        h = self.Nph // 2
        across = self._roll(u, h, 1)  # the meridian at phi + pi
        if self.xp is np:
            up = np.concatenate([across[:1], u[:-1]], axis=0)    # u[j-1]; j = 0 reads across the north pole
            dn = np.concatenate([u[1:], across[-1:]], axis=0)    # u[j+1]; j = Nth-1 reads across the south pole
        else:
            up = self.xp.cat([across[:1], u[:-1]], dim=0)
            dn = self.xp.cat([u[1:], across[-1:]], dim=0)
        dudth = (dn - up) / (2 * self.dth)
        dudph = (self._roll(u, -1, 1) - self._roll(u, 1, 1)) / (2 * self.dph)
        return self.a * dudth + self.b * dudph

    def cfl_steps(self) -> tuple:
        """(theta limit, axis limit) of the SSP-RK3 step for centred differences (imaginary-axis
        stability bound sqrt(3) over the largest |coefficient| / spacing)."""
        r3 = math.sqrt(3.0)
        th0 = 0.5 * self.dth
        return r3 * self.dth / self.omega, r3 * self.dph * math.tan(th0) / self.omega


def ssp_rk3_step(u, dt: float, rhs: Callable, filt: Filter | None):
    """One SSP-RK3 step with the filter applied after every substep (when given)."""
    f = filt if filt is not None else (lambda v: v)
    u1 = f(u + dt * rhs(u))
    u2 = f(0.75 * u + 0.25 * (u1 + dt * rhs(u1)))
    return f(u / 3.0 + (2.0 / 3.0) * (u2 + dt * rhs(u2)))


def blob(Ntheta: int, Nphi: int, centre=(math.pi / 3, 0.5), width: float = 0.35) -> np.ndarray:
    """A smooth Gaussian bump on the sphere (great-circle distance from `centre`)."""
    th = (np.arange(Ntheta) + 0.5) * math.pi / Ntheta
    ph = 2 * math.pi * np.arange(Nphi) / Nphi
    t0, p0 = centre
    cosd = (np.sin(th)[:, None] * math.sin(t0) * np.cos(ph[None, :] - p0) + np.cos(th)[:, None] * math.cos(t0))
    d = np.arccos(np.clip(cosd, -1.0, 1.0))
    return np.exp(-(d / width) ** 2)


def plan_filter(Ntheta: int, Nphi: int, L: float = 1.0, kind: int = 2, precision: int = 2):
    """The filter of this package for one scalar (even parity) on one shell, as a callable on
    [Ntheta, Nphi] CUDA tensors. The shell radius is set so that m_max reaches the Nyquist mode at
    the equator (2 r / dr_min L = Nphi / 2): only the rings near the axis are filtered."""
    from .binding import Plan
    from . import workloads as W
    r = Nphi / (4.0 * L)
    g = W.Grid(1, Ntheta, Nphi, [0], [kind], [L], np.array([r]), dr_min=1.0, floor=2.0)
    plan = Plan.from_grid(g, precision=precision)

    def filt(u):
        return plan.apply(u.reshape(1, 1, Ntheta, Nphi).contiguous()).reshape(Ntheta, Nphi)

    filt.plan = plan
    return filt


def run(u0, steps: int, dt: float, problem: RotationAdvection, filt: Filter | None):
    """Advance u0 by `steps` SSP-RK3 steps; returns the final field and the max |u| after each
    step (as floats)."""
    u = u0
    peaks = []
    for _ in range(steps):
        u = ssp_rk3_step(u, dt, problem.rhs, filt)
        peaks.append(float(abs(u).max()))
    return u, peaks
