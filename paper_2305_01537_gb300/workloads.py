"""Seeded synthetic workloads for the double FFT filter.

This module only makes inputs: grid shapes, the per-field parameter mix and random fields. It
holds none of the filter's arithmetic, so the oracle and the CUDA path can both consume it.

Grids: theta_j = (j + 1/2) pi / Ntheta (cell centred, no point on a pole), phi_k = 2 pi k / Nphi,
shell radii r_i = i + 1/2 with dr_min = 1 (no fisheye map), cutoff floor 2.

Fields are random sums of parity-consistent angular modes cos/sin(m phi) * P_l(theta) with
P_l = cos(l theta) when (a + m) is even and sin(l theta) (l >= 1) when (a + m) is odd, a being
the field's parity across the pole. Such a mode continues smoothly over the pole in the paper's
double covering (Sec. II.C), as a smooth field of that parity does. White noise (uniform) is
added at every grid point, so every Fourier mode carries power.

The 28-field mix follows the paper's field classes (Sec. II.C): exponential filter with L = 3
for spacetime fields, Gaussian with L = 12 for D, S_i, tau, entropy and exponential with L = 12
for A_i and Phi. The parity split (20 even / 8 odd) is an assumption; the paper defers it to a
table of another paper. The hybrid mix gives the six matter fields the hybrid filter instead of
the Gaussian (Sec. II.C: exponential unless Jameson's detector finds a discontinuity), on a "star"
state whose matter fields drop from O(1) to an atmosphere of 1e-10 across a sphere's surface.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

EXP, GAUSS, SHARP, HYBRID = 0, 1, 2, 3


@dataclass
class Grid:
    """One spherical grid and its filter parameters (everything the plan needs)."""
    Nr: int
    Ntheta: int
    Nphi: int
    parity: List[int]
    kind: List[int]
    L: List[float]
    r: np.ndarray = None
    dr_min: float = 1.0
    floor: float = 2.0
    eps: float = 1e-12  # epsilon of Jameson's detector (hybrid fields)

    def __post_init__(self):
        if self.r is None:
            self.r = np.arange(self.Nr, dtype=np.float64) + 0.5

    @property
    def nvars(self) -> int:
        return len(self.parity)

    @property
    def shape(self):
        return (self.nvars, self.Nr, self.Ntheta, self.Nphi)

    @property
    def points(self) -> int:
        return self.nvars * self.Nr * self.Ntheta * self.Nphi


def field_mix_28():
    """(parity, kind, L) for the 28-field spacetime + GRMHD mix."""
    parity, kind, L = [], [], []
    # 20 even fields
    parity += [0] * 14; kind += [EXP] * 14; L += [3.0] * 14          # spacetime scalars / diagonal
    parity += [0] * 4; kind += [GAUSS] * 4; L += [12.0] * 4         # D, tau, S_r, entropy
    parity += [0] * 2; kind += [EXP] * 2; L += [12.0] * 2           # A_r, Phi
    # 8 odd fields (theta/phi vector components)
    parity += [1] * 4; kind += [EXP] * 4; L += [3.0] * 4            # theta/phi spacetime comps
    parity += [1] * 2; kind += [GAUSS] * 2; L += [12.0] * 2         # S_theta, S_phi
    parity += [1] * 2; kind += [EXP] * 2; L += [12.0] * 2           # A_theta, A_phi
    return parity, kind, L


def field_mix_28_hybrid():
    """The 28-field mix with the six matter fields (Gaussian in field_mix_28) on the hybrid filter."""
    parity, kind, L = field_mix_28()
    return parity, [HYBRID if k == GAUSS else k for k in kind], L


def field_mix_8():
    """Eight-field mix of the differentiable chain: 6 even and 2 odd, exponential, L = 3."""
    return [0] * 6 + [1] * 2, [EXP] * 8, [3.0] * 8


def grid_28(Nr, Nth, Nph) -> Grid:
    p, k, L = field_mix_28()
    return Grid(Nr, Nth, Nph, p, k, L)


def grid_28_hybrid(Nr, Nth, Nph) -> Grid:
    p, k, L = field_mix_28_hybrid()
    return Grid(Nr, Nth, Nph, p, k, L)


def theta_points(Nth):
    return (np.arange(Nth, dtype=np.float64) + 0.5) * np.pi / Nth


def phi_points(Nph):
    return 2.0 * np.pi * np.arange(Nph, dtype=np.float64) / Nph


def _mode_sum(parity_of_shell, amp_c, amp_s, Nth, Nph):
    """x[s, j, k] = sum_{l, m} (amp_c[s,l,m] cos(m phi_k) + amp_s[s,l,m] sin(m phi_k)) P_l^{(a_s+m)}(theta_j)."""
    S, Lp1, Mp1 = amp_c.shape
    th = theta_points(Nth)
    ph = phi_points(Nph)
    l = np.arange(Lp1)
    m = np.arange(Mp1)
    Pc = np.cos(np.outer(th, l))                  # [Nth, L+1]
    Ps = np.sin(np.outer(th, l))                  # l = 0 column is zero
    odd = ((parity_of_shell[:, None] + m[None, :]) % 2).astype(np.float64)[:, None, :]  # [S,1,M+1]
    Bc = np.einsum("jl,slm->sjm", Pc, amp_c) * (1 - odd) + np.einsum("jl,slm->sjm", Ps, amp_c) * odd
    Bs = np.einsum("jl,slm->sjm", Pc, amp_s) * (1 - odd) + np.einsum("jl,slm->sjm", Ps, amp_s) * odd
    C = np.cos(np.outer(m, ph))                   # [M+1, Nph]
    Sn = np.sin(np.outer(m, ph))
    return Bc @ C + Bs @ Sn


def band_limited_state(grid: Grid, seed: int, mode_max: int, noise: float,
                       chunk_shells: int = 1024) -> np.ndarray:
    """Random smooth part with all modes l, m <= mode_max (N(0,1) amplitudes, both phi phases)
    plus U(-noise, noise) at every point. Returns float64 [nvars][Nr][Ntheta][Nphi]."""
    rng = np.random.default_rng(seed)
    S = grid.nvars * grid.Nr
    amp_c = rng.standard_normal((S, mode_max + 1, mode_max + 1))
    amp_s = rng.standard_normal((S, mode_max + 1, mode_max + 1))
    shell_parity = np.repeat(np.asarray(grid.parity), grid.Nr)
    out = np.empty((S, grid.Ntheta, grid.Nphi), dtype=np.float64)
    for s0 in range(0, S, chunk_shells):
        s1 = min(S, s0 + chunk_shells)
        out[s0:s1] = _mode_sum(shell_parity[s0:s1], amp_c[s0:s1], amp_s[s0:s1], grid.Ntheta, grid.Nphi)
        out[s0:s1] += rng.uniform(-noise, noise, size=(s1 - s0, grid.Ntheta, grid.Nphi))
    return out.reshape(grid.shape)


def star_state(grid: Grid, seed: int, mode_max: int = 4, noise: float = 0.05, centre_r: float = None,
               radius: float = None) -> np.ndarray:
    """Fields of hybrid kind get a "star": rho = 1 inside a ball, 1e-10 (atmosphere) outside, times a
    smooth factor: rho (1 + g / 2) for even fields, rho g for odd ones, g a random band-limited
    field of that parity (modes l, m <= mode_max) scaled to max |g| = 1. The ball has radius
    `radius` (default 0.234 Nr) around the point at radius `centre_r` (default 0.3125 Nr),
    theta = pi/3, phi = 0.5, so that with shells r = i + 1/2 the middle shells cut its surface.
    The other fields are band_limited_state(mode_max = Nphi / 8, noise). No noise on the star
    fields: their smooth parts keep Jameson's sigma small."""
    x = band_limited_state(grid, seed, mode_max=max(1, grid.Nphi // 8), noise=noise)
    hyb = [v for v in range(grid.nvars) if grid.kind[v] == HYBRID]
    if not hyb:
        return x
    th, ph = theta_points(grid.Ntheta), phi_points(grid.Nphi)
    r = np.asarray(grid.r, dtype=np.float64)
    st, ct = np.sin(th)[None, :, None], np.cos(th)[None, :, None]
    sp, cp = np.sin(ph)[None, None, :], np.cos(ph)[None, None, :]
    rr = r[:, None, None]
    X, Y, Z = rr * st * cp, rr * st * sp, rr * ct * np.ones_like(cp)
    rc = 0.3125 * grid.Nr if centre_r is None else centre_r
    R = 0.234375 * grid.Nr if radius is None else radius
    tc, pc = np.pi / 3, 0.5
    cx, cy, cz = rc * np.sin(tc) * np.cos(pc), rc * np.sin(tc) * np.sin(pc), rc * np.cos(tc)
    rho = np.where((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 < R * R, 1.0, 1e-10)
    rng = np.random.default_rng([seed, 2])
    for v in hyb:
        amp_c = rng.standard_normal((grid.Nr, mode_max + 1, mode_max + 1))
        amp_s = rng.standard_normal((grid.Nr, mode_max + 1, mode_max + 1))
        g = _mode_sum(np.full(grid.Nr, grid.parity[v]), amp_c, amp_s, grid.Ntheta, grid.Nphi)
        g /= np.abs(g).max(axis=(1, 2), keepdims=True)
        x[v] = rho * (g if grid.parity[v] else 1.0 + 0.5 * g)
    return x


def few_mode_state(grid: Grid, seed: int, nmodes: int, mode_max: int, noise: float) -> np.ndarray:
    """Per shell, a sum of `nmodes` random modes: m, l ~ U{0..mode_max} (l >= 1 for the sin profile),
    cos or sin in phi with probability 1/2, N(0,1) amplitude; plus U(-noise, noise) per point."""
    rng = np.random.default_rng(seed)
    S = grid.nvars * grid.Nr
    shell_parity = np.repeat(np.asarray(grid.parity), grid.Nr)
    amp_c = np.zeros((S, mode_max + 1, mode_max + 1))
    amp_s = np.zeros((S, mode_max + 1, mode_max + 1))
    for s in range(S):
        for _ in range(nmodes):
            m = int(rng.integers(0, mode_max + 1))
            if (shell_parity[s] + m) % 2 == 1:
                l = int(rng.integers(1, mode_max + 1))
            else:
                l = int(rng.integers(0, mode_max + 1))
            a = rng.standard_normal()
            if rng.random() < 0.5:
                amp_c[s, l, m] += a
            else:
                amp_s[s, l, m] += a
    x = _mode_sum(shell_parity, amp_c, amp_s, grid.Ntheta, grid.Nphi)
    x += rng.uniform(-noise, noise, size=x.shape)
    return x.reshape(grid.shape)


# ---------------------------------------------------------------------------------------------
# The named workloads. Each returns (grid(s), state(s)); sizes and seeds are fixed.

@dataclass
class Workload:
    name: str
    grids: List[Grid]
    seeds: List[int]
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return sum(g.points for g in self.grids)

    def state(self, index: int = 0) -> np.ndarray:
        g = self.grids[index]
        seed = self.seeds[index]
        if self.name == "single_field_16x16x32":
            return few_mode_state(g, seed, nmodes=6, mode_max=4, noise=1e-3)
        if self.name.startswith("hybrid28_"):
            return star_state(g, seed)
        return band_limited_state(g, seed, mode_max=g.Nphi // 8, noise=0.05)


def single_field() -> Workload:
    """1 even scalar, exponential filter L = 3, Nr = 16, Ntheta = 16, Nphi = 32, seed 0."""
    g = Grid(16, 16, 32, [0], [EXP], [3.0])
    return Workload("single_field_16x16x32", [g], [0], "1 even exp-L3 field, 6 low modes + 1e-3 noise")


def full_state_128x64x128() -> Workload:
    """28 mixed-parity fields, Nr = 128, Ntheta = 64, Nphi = 128, seed 1."""
    return Workload("state28_128x64x128", [grid_28(128, 64, 128)], [1],
                    "28 mixed-parity fields, band-limited m,l<=16 + U(-0.05,0.05)")


def full_state_256x128x256() -> Workload:
    """28 mixed-parity fields, Nr = 256, Ntheta = 128, Nphi = 256, seed 2."""
    return Workload("state28_256x128x256", [grid_28(256, 128, 256)], [2],
                    "28 mixed-parity fields, band-limited m,l<=32 + U(-0.05,0.05)")


def state_32x128x256() -> Workload:
    """The 128 x 256 shells of the 256 x 128 x 256 workload at its first 32 radii (r = 0.5 .. 31.5):
    28 fields, Nr = 32, seed 2; a case small enough for detailed profiles of the 128 x 256 kernels."""
    return Workload("state28_32x128x256", [grid_28(32, 128, 256)], [2],
                    "28 mixed-parity fields, band-limited m,l<=32 + U(-0.05,0.05)")


def hybrid_state_128x64x128() -> Workload:
    """The 28-field mix with hybrid-filtered matter fields on a star state, Nr = 128, Ntheta = 64,
    Nphi = 128, seed 10."""
    return Workload("hybrid28_128x64x128", [grid_28_hybrid(128, 64, 128)], [10],
                    "28 fields, 6 hybrid matter fields with a star surface (1 -> 1e-10), others band-limited")


def hybrid_state_256x128x256() -> Workload:
    """The hybrid 28-field mix on Nr = 256, Ntheta = 128, Nphi = 256 (CTA pairs), seed 11."""
    return Workload("hybrid28_256x128x256", [grid_28_hybrid(256, 128, 256)], [11],
                    "28 fields, 6 hybrid matter fields with a star surface (1 -> 1e-10), others band-limited")


def hybrid_state_32x128x256() -> Workload:
    """The hybrid 28-field mix on the 128 x 256 shells at 32 radii (r = 0.5 .. 31.5, the star's
    surface crossing r = 2.5 .. 17.5), seed 12: a case small enough for detailed profiles of the
    CTA-pair kernel's hybrid variant."""
    return Workload("hybrid28_32x128x256", [grid_28_hybrid(32, 128, 256)], [12],
                    "28 fields, 6 hybrid matter fields with a star surface (1 -> 1e-10), others band-limited")


BATCH_SHAPES = [(16, 32, 64), (32, 64, 96), (48, 96, 128), (64, 128, 256), (96, 192, 384), (128, 256, 512)]


def batched_six_grids() -> Workload:
    """Six independent grids (Ntheta, Nphi, Nr), 28 fields each, seeds 3..8."""
    grids = [grid_28(Nr, Nth, Nph) for (Nth, Nph, Nr) in BATCH_SHAPES]
    return Workload("batch6_uneven", grids, [3, 4, 5, 6, 7, 8],
                    "6 uneven grids x 28 fields, 3 applications per step")


def chain_8field() -> Workload:
    """8 fields (6 even, 2 odd, exponential L = 3), Nr = 128, Ntheta = 64, Nphi = 128, seed 9."""
    p, k, L = field_mix_8()
    return Workload("chain8_128x64x128", [Grid(128, 64, 128, p, k, L)], [9],
                    "8 chained filters with tanh between, loss sum w*y^2")


def chain_weights(grid: Grid, seed: int = 9) -> np.ndarray:
    """Loss weights w ~ U(0, 1), drawn from a stream separate from the state's."""
    rng = np.random.default_rng([seed, 1])
    return rng.uniform(0.0, 1.0, size=grid.shape)


def random_state(shape: Sequence[int], seed: int) -> np.ndarray:
    """Plain N(0,1) state of the given shape (for invariants and adjoint identities)."""
    return np.random.default_rng(seed).standard_normal(tuple(shape))
