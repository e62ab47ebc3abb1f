"""Seeded synthetic initial conditions shaped like the paper's test problems.

This module only draws marker positions, velocities and weights from the
initial distributions; it holds none of the scheme's arithmetic (no shapes,
no push, no field solve), so it can feed both the CUDA library and the CPU
oracle with identical arrays.  All generators use numpy's PCG64 with an
explicit seed.

Dimensionless units of Sec. 2.1 (time in 1/omega_p, length in Debye lengths,
velocity in thermal speeds); electrons have q = -1, m = 1 over a fixed,
uniform, neutralising ion background of density 1, so the marker weight is
w = n0 L / N with n0 = 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Markers1D:
    q: float
    m: float
    x: np.ndarray          # float64 [n], in [0, L)
    v: np.ndarray          # float64 [n]
    w: Optional[np.ndarray] = None   # float64 [n] or None (uniform w0)
    w0: float = 0.0


@dataclass
class Problem1D:
    name: str
    L: float
    nc: int
    order: int
    dt: float
    steps: int
    species: List[Markers1D] = field(default_factory=list)

    @property
    def n_markers(self) -> int:
        return sum(len(s.x) for s in self.species)


def sample_cosine_density(rng: np.random.Generator, n: int, L: float, k: float, alpha: float,
                          quiet: bool = False) -> np.ndarray:
    """Positions on [0, L) with density proportional to 1 + alpha cos(k x).

    Inverse-CDF sampling: F(x) = (x + (alpha/k) sin(k x)) / L is inverted by
    Newton's method from uniform (or, with quiet=True, evenly spaced) u.
    """
    if quiet:
        u = (np.arange(n, dtype=np.float64) + 0.5) / n
    else:
        u = rng.random(n)
    target = u * L
    x = target.copy()
    for _ in range(60):
        f = x + (alpha / k) * np.sin(k * x) - target
        fp = 1.0 + alpha * np.cos(k * x)
        dx = f / fp
        x -= dx
        if np.max(np.abs(dx)) < 1e-15 * L:
            break
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return x


def gaussian_quantiles(nv: int) -> np.ndarray:
    """Standard-normal quantiles at the cell centres (j + 1/2)/nv, j = 0..nv-1."""
    from scipy.special import ndtri
    return ndtri((np.arange(nv, dtype=np.float64) + 0.5) / nv)


def phase_space_lattice(nx: int, nv: int, L: float, k: float, alpha: float):
    """Quiet start: every one of nx evenly spaced density quantiles of 1 + alpha cos kx
    carries the same nv Gaussian velocity quantiles (no velocity noise)."""
    u = (np.arange(nx, dtype=np.float64) + 0.5) / nx
    target = u * L
    x = target.copy()
    for _ in range(60):
        dx = (x + (alpha / k) * np.sin(k * x) - target) / (1.0 + alpha * np.cos(k * x))
        x -= dx
        if np.max(np.abs(dx)) < 1e-15 * L:
            break
    vq = gaussian_quantiles(nv)
    X = np.repeat(x, nv)
    V = np.tile(vq, nx)
    return X, V


def landau(n: int = 20_000, nc: int = 64, k: float = 0.5, alpha: float = 0.01,
           vth: float = 1.0, dt: float = 0.1, steps: int = 200, order: int = 1,
           seed: int = 0, quiet: bool = False, lattice_nv: int = 0,
           lattice_vmax: float = 6.0) -> Problem1D:
    """1D1V linear Landau damping: f0 = (1 + alpha cos kx) exp(-v^2/2 vth^2)/sqrt(2 pi) vth,
    L = 2 pi / k (the 1D restatement of the paper's Sec. 5.1 test).

    lattice_nv > 0 selects a noise-free weighted lattice: n // lattice_nv evenly
    spaced density quantiles, each carrying lattice_nv velocities on a uniform grid
    of [-vmax, vmax] vth with weights proportional to the Maxwellian (the resonant
    tail is sampled as finely as the bulk)."""
    rng = np.random.default_rng(seed)
    L = 2.0 * np.pi / k
    if lattice_nv:
        nx = n // lattice_nv
        xq, _ = phase_space_lattice(nx, 1, L, k, alpha)
        dv = 2.0 * lattice_vmax / lattice_nv
        vg = -lattice_vmax + (np.arange(lattice_nv) + 0.5) * dv
        fv = np.exp(-0.5 * vg * vg)
        fv = fv / fv.sum()
        x = np.repeat(xq, lattice_nv)
        v = np.tile(vg, nx) * vth
        w = np.tile(fv, nx) * (L / nx)
        return Problem1D("landau", L, nc, order, dt, steps,
                         [Markers1D(-1.0, 1.0, x, v, w, 0.0)])
    x = sample_cosine_density(rng, n, L, k, alpha, quiet)
    v = rng.standard_normal(n) * vth
    return Problem1D("landau", L, nc, order, dt, steps,
                     [Markers1D(-1.0, 1.0, x, v, None, L / n)])


def two_stream(n: int = 1 << 23, nc: int = 512, k: float = 0.2, v0: float = 3.0,
               vth: float = 0.1, alpha: float = 1e-3, dt: float = 0.05, steps: int = 2000,
               order: int = 2, seed: int = 0, quiet: bool = False,
               lattice_nv: int = 0) -> Problem1D:
    """1D1V two-stream instability: two beams at +-v0 (half the markers each) with
    thermal spread vth and density 1 + alpha cos kx, L = 2 pi / k (1D restatement of
    Sec. 5.2).  lattice_nv > 0 selects the noise-free phase-space lattice."""
    rng = np.random.default_rng(seed)
    L = 2.0 * np.pi / k
    if lattice_nv:
        x, vq = phase_space_lattice(n // (2 * lattice_nv), lattice_nv, L, k, alpha)
        x = np.concatenate([x, x])
        v = np.concatenate([v0 + vth * vq, -v0 + vth * vq])
        n = len(x)
    else:
        x = sample_cosine_density(rng, n, L, k, alpha, quiet)
        sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
        v = sign * v0 + rng.standard_normal(n) * vth
    return Problem1D("two_stream", L, nc, order, dt, steps,
                     [Markers1D(-1.0, 1.0, x, v, None, L / n)])


def ensemble(nruns: int = 256, seed: int = 0, n_min: float = 1e4, n_max: float = 1e6,
             nc_min: int = 32, nc_max: int = 512):
    """Independent 1D1V problems for a batched run: per run N_c ~ U{nc_min..nc_max},
    N ~ log-uniform on [n_min, n_max], seed amplitude alpha ~ U[1e-3, 0.1]; even runs
    Landau damping (CIC, dt 0.1), odd runs two-stream (quadratic shapes, dt 0.05)."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(nruns):
        nc = int(rng.integers(nc_min, nc_max + 1))
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        alpha = float(rng.uniform(1e-3, 0.1))
        s = int(rng.integers(0, 2**31 - 1))
        if r % 2 == 0:
            runs.append(landau(n=n, nc=nc, alpha=alpha, seed=s))
        else:
            runs.append(two_stream(n=n, nc=nc, alpha=alpha, seed=s))
    return runs


def bump_on_tail(n: int = 1 << 20, nc: int = 256, k: float = 0.3, alpha: float = 0.04,
                 beam_frac: float = 0.1, vb: float = 4.5, vtb: float = 0.5,
                 dt: float = 0.1, steps: int = 500, order: int = 2, seed: int = 0) -> Problem1D:
    """1D1V bump-on-tail with weighted markers: x uniform on L = 20 pi, v from
    0.9 N(0,1) + 0.1 N(vb, vtb^2), weights w_p = (L/N)(1 + alpha cos k x_p)."""
    rng = np.random.default_rng(seed)
    L = 20.0 * np.pi
    x = rng.random(n) * L
    beam = rng.random(n) < beam_frac
    v = np.where(beam, vb + vtb * rng.standard_normal(n), rng.standard_normal(n))
    w = (L / n) * (1.0 + alpha * np.cos(k * x))
    return Problem1D("bump_on_tail", L, nc, order, dt, steps,
                     [Markers1D(-1.0, 1.0, x, v, w, 0.0)])


def cold_oscillation(n: int = 4096, nc: int = 32, L: float = 2 * np.pi, amp: float = 1e-3,
                     dt: float = 0.05, order: int = 1) -> Problem1D:
    """Cold, evenly spaced electrons with a small sinusoidal velocity kick
    v = amp sin(2 pi x / L): the plasma oscillates at omega_p = 1."""
    x = (np.arange(n, dtype=np.float64) + 0.5) * (L / n)
    v = amp * np.sin(2 * np.pi * x / L)
    return Problem1D("cold_oscillation", L, nc, order, dt, 0,
                     [Markers1D(-1.0, 1.0, x, v, None, L / n)])


# ----------------------------------------------------------------------------- 2D3V


@dataclass
class Markers2D:
    q: float
    m: float
    x: np.ndarray
    y: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    w: Optional[np.ndarray] = None
    w0: float = 0.0


@dataclass
class Problem2D:
    name: str
    nx: int
    ny: int
    Lx: float
    Ly: float
    order: int
    dt: float
    c: float
    steps: int
    species: List[Markers2D] = field(default_factory=list)

    @property
    def n_markers(self) -> int:
        return sum(len(s.x) for s in self.species)


def weibel(nx: int = 128, ny: int = 128, ppc: int = 64, L: float = 12.8, vth_par: float = 0.05,
           t_ratio: float = 10.0, c: float = 1.0, cfl: float = 0.5, steps: int = 4000,
           order: int = 1, seed: int = 0, quiet: bool = False,
           mirrored: bool = False) -> Problem2D:
    """2D3V Weibel instability: uniform electrons, bi-Maxwellian with vth_par along x
    and sqrt(t_ratio) vth_par along y and z; dt from c dt sqrt(hx^-2 + hy^-2) = cfl.
    quiet: positions on a lattice of about ppc points per cell.  mirrored (with
    quiet): the markers come in eights at one point with the eight sign patterns
    of one drawn velocity, so no cell carries current at the start."""
    rng = np.random.default_rng(seed)
    n = nx * ny * ppc
    hx, hy = L / nx, L / ny
    dt = cfl / (c * np.sqrt(hx ** -2 + hy ** -2))
    if quiet:
        per = ppc // 8 if mirrored else ppc
        side = int(round(np.sqrt(per)))
        gx = (np.arange(nx * side) + 0.5) * (L / (nx * side))
        gy = (np.arange(ny * side) + 0.5) * (L / (ny * side))
        X, Y = np.meshgrid(gx, gy)
        x, y = X.ravel().copy(), Y.ravel().copy()
        n = len(x)
    else:
        x = rng.random(n) * L
        y = rng.random(n) * L
    vperp = vth_par * np.sqrt(t_ratio)
    vx = rng.standard_normal(n) * vth_par
    vy = rng.standard_normal(n) * vperp
    vz = rng.standard_normal(n) * vperp
    if quiet and mirrored:
        sx, sy, sz = (np.array([(k >> b & 1) * -2 + 1 for k in range(8)], dtype=float)
                      for b in range(3))
        x, y = np.repeat(x, 8), np.repeat(y, 8)
        vx = (vx[:, None] * sx).ravel()
        vy = (vy[:, None] * sy).ravel()
        vz = (vz[:, None] * sz).ravel()
        n = len(x)
    return Problem2D("weibel", nx, ny, L, L, order, dt, c, steps,
                     [Markers2D(-1.0, 1.0, x, y, vx, vy, vz, None, L * L / n)])


@dataclass
class Markers1D2V:
    q: float
    m: float
    y: np.ndarray          # float64 [n], in [0, L)
    vx: np.ndarray
    vy: np.ndarray
    w: Optional[np.ndarray] = None
    w0: float = 0.0


@dataclass
class Problem1D2V:
    """1D2V electromagnetic problem: coordinate y, velocities (vx, vy), fields
    E = (Ex, Ey) [2, n] and Bz [n] on n collocated nodes."""
    name: str
    L: float
    n: int
    order: int
    dt: float
    c: float
    steps: int
    E0: np.ndarray
    B0: np.ndarray
    species: List[Markers1D2V] = field(default_factory=list)

    @property
    def n_markers(self) -> int:
        return sum(len(s.y) for s in self.species)


def weibel_1d2v(n: int = 32, ppc: int = 3200, k0: float = 0.2, beta: float = 0.01,
                delta: float = 0.5, v01: float = 0.3, v02: float = 0.3, b: float = 0.001,
                dt: float = 0.1, c: float = 1.0, steps: int = 1000, order: int = 1,
                mirrored: bool = False, seed: int = 0) -> Problem1D2V:
    """The Weibel test of Sec. 5 (Exp. 3): L = 2 pi / k0, quiet start (markers
    evenly spaced in y), f ~ exp(-vy^2/beta) [delta exp(-(vx - v01)^2/beta)
    + (1 - delta) exp(-(vx + v02)^2/beta)], E = 0, Bz = b sin(k0 y).
    mirrored: markers come in fours (vx, vy), (-vx, -vy), (vx, -vy), (-vx, vy)
    at the same y (only for delta = 1/2 and v01 = v02). Free streaming then
    deposits no jx at any time, so only the seed b drives (Ex, Bz)."""
    rng = np.random.default_rng(seed)
    L = 2.0 * np.pi / k0
    N = n * ppc
    y = (np.arange(N) + 0.5) * (L / N)
    sd = np.sqrt(beta / 2.0)
    if mirrored:
        assert N % 4 == 0 and delta == 0.5 and v01 == v02
        q = N // 4
        ax = np.where(rng.random(q) < delta, v01, -v02) + sd * rng.standard_normal(q)
        ay = sd * rng.standard_normal(q)
        vx = np.stack([ax, -ax, ax, -ax], axis=1).ravel()
        vy = np.stack([ay, -ay, -ay, ay], axis=1).ravel()
        y = np.repeat((np.arange(q) + 0.5) * (L / q), 4)
    else:
        beam = np.where(rng.random(N) < delta, v01, -v02)
        vx = beam + sd * rng.standard_normal(N)
        vy = sd * rng.standard_normal(N)
    nodes = np.arange(n) * (L / n)
    E0 = np.zeros((2, n))
    B0 = b * np.sin(k0 * nodes)
    return Problem1D2V("weibel_1d2v", L, n, order, dt, c, steps, E0, B0,
                       [Markers1D2V(-1.0, 1.0, y, vx, vy, None, L / N)])
