"""Seeded synthetic plasma workloads.

This module only draws inputs: particle positions, momenta, weights and the
initial fields of each workload.  It holds none of the particle-in-cell
arithmetic; the CUDA path and the CPU oracle both consume what it returns.

Units are normalised to a reference frequency w_r: time 1/w_r, length c/w_r,
momentum u = gamma v / c, fields m c w_r / e, density n_r = m w_r^2/(4 pi e^2).
A macro-particle's weight is its number of real particles in these units,
w = n dV / ppc.

The workloads mirror the paper's "frozen plasma" benchmark (arXiv:1608.01009,
Sec. 3: a 40^3 grid, 50 particles per cell, double precision, cloud-in-cell,
Villasenor-Buneman), which the paper does not define further; it is read here
as a uniform periodic thermal electron plasma over an immobile neutralising
ion background.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

PERIODIC = 0
ABSORBING = 1


@dataclass
class Species:
    q: float
    m: float
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def arrays(self):
        return [self.x, self.y, self.z, self.ux, self.uy, self.uz, self.w]

    def copy(self) -> "Species":
        return Species(self.q, self.m, *[a.copy() for a in self.arrays()])


@dataclass
class Workload:
    name: str
    n: Tuple[int, int, int]
    d: Tuple[float, float, float]
    dt: float
    steps: int
    species: List[Species]
    E: np.ndarray  # (3, nz, ny, nx): x fastest in each component
    B: np.ndarray
    bc: Tuple[int, int, int] = (PERIODIC, PERIODIC, PERIODIC)
    absorb_cells: int = 8
    absorb_sigma: float = 0.1
    meta: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def nparticles(self) -> int:
        return sum(s.n for s in self.species)

    def copy(self) -> "Workload":
        return Workload(self.name, self.n, self.d, self.dt, self.steps,
                        [s.copy() for s in self.species], self.E.copy(), self.B.copy(),
                        self.bc, self.absorb_cells, self.absorb_sigma, dict(self.meta))


def courant_dt(d, factor: float = 0.5) -> float:
    """dt = factor * delta / (c sqrt(3)) for a cubic cell (the configs' rule)."""
    return factor * min(d) / math.sqrt(3.0)


def _cells_repeated(n, ppc, region=None):
    nx, ny, nz = n
    if region is None:
        region = ((0, nx), (0, ny), (0, nz))
    (x0, x1), (y0, y1), (z0, z1) = region
    kk, jj, ii = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    return np.repeat(cells, ppc, axis=0)


def uniform_plasma(n=(16, 16, 16), ppc=8, delta=0.05, vth=0.05, density=1.0, seed=1234,
                   perturb_eps: float = 0.0, steps=50, name="uniform", dt_factor=0.5,
                   q=-1.0, m=1.0) -> Workload:
    """Uniform periodic thermal electron plasma, ppc electrons drawn uniformly in
    every cell, each momentum component vth * N(0, 1), zero initial fields.
    delta: the cell size, one value (cubic cells) or one per axis.

    perturb_eps > 0 displaces x by (eps / k) cos(k x) with k = 2 pi / Lx
    (mode 1), which gives a density n (1 + eps sin k x) to first order.
    """
    rng = np.random.default_rng(seed)
    d = tuple(float(v) for v in np.broadcast_to(np.asarray(delta, dtype=np.float64), (3,)))
    cells = _cells_repeated(n, ppc)
    npart = cells.shape[0]
    pos = (cells + rng.random((npart, 3))) * np.array(d)
    if perturb_eps:
        Lx = n[0] * d[0]
        k = 2.0 * math.pi / Lx
        x = pos[:, 0] + (perturb_eps / k) * np.cos(k * pos[:, 0])
        pos[:, 0] = np.mod(x, Lx)
    u = vth * rng.standard_normal((npart, 3))
    w = np.full(npart, density * d[0] * d[1] * d[2] / ppc)
    sp = Species(q, m, pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(),
                 u[:, 0].copy(), u[:, 1].copy(), u[:, 2].copy(), w)
    shape = (3, n[2], n[1], n[0])
    return Workload(name, tuple(n), d, courant_dt(d, dt_factor), steps, [sp],
                    np.zeros(shape), np.zeros(shape),
                    meta=dict(ppc=ppc, vth=vth, density=density, seed=seed, perturb_eps=perturb_eps))


def _stag(comp: int, axis: int, magnetic: bool) -> float:
    """Lattice offset (in cells) of a Yee component along an axis."""
    if magnetic:
        return 0.0 if comp == axis else 0.5
    return 0.5 if comp == axis else 0.0


def _positions(n, d, comp, magnetic):
    nx, ny, nz = n
    zz, yy, xx = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                             np.arange(nx, dtype=np.float64), indexing="ij")
    return ((xx + _stag(comp, 0, magnetic)) * d[0], (yy + _stag(comp, 1, magnetic)) * d[1],
            (zz + _stag(comp, 2, magnetic)) * d[2])


def laser_slab(n=(32, 32, 64), ppc=16, slab=(24, 40), density=0.1, a0=1.0, wavelength_cells=16,
               window=(4, 20), seed=1238, steps=200, name="laser_slab") -> Workload:
    """Cold electron slab z in [slab) cells at `density` n_crit, periodic in x/y
    and absorbing in z, with a +z plane wave Ex = By = a0 sin(k(z - z0)) env(z)
    whose sin^2 envelope spans the `window` cells (one wavelength), each
    component sampled at its own staggered position at t = 0."""
    rng = np.random.default_rng(seed)
    delta = 2.0 * math.pi / wavelength_cells  # w_r = w_L, wavelength = 2 pi c / w_L
    d = (delta, delta, delta)
    cells = _cells_repeated(n, ppc, ((0, n[0]), (0, n[1]), (slab[0], slab[1])))
    npart = cells.shape[0]
    pos = (cells + rng.random((npart, 3))) * delta
    zero = np.zeros(npart)
    w = np.full(npart, density * delta ** 3 / ppc)
    sp = Species(-1.0, 1.0, pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(), zero.copy(),
                 zero.copy(), zero.copy(), w)
    shape = (3, n[2], n[1], n[0])
    E = np.zeros(shape)
    B = np.zeros(shape)
    k = 2.0 * math.pi / (wavelength_cells * delta)
    z0, z1 = window[0] * delta, window[1] * delta

    def profile(z):
        env = np.where((z >= z0) & (z < z1), np.sin(math.pi * (z - z0) / (z1 - z0)) ** 2, 0.0)
        return a0 * np.sin(k * (z - z0)) * env

    E[0] = profile(_positions(n, d, 0, False)[2])
    B[1] = profile(_positions(n, d, 1, True)[2])
    return Workload(name, tuple(n), d, courant_dt(d), steps, [sp], E, B,
                    bc=(PERIODIC, PERIODIC, ABSORBING),
                    meta=dict(ppc=ppc, a0=a0, density=density, seed=seed, slab=slab, window=window,
                              wavelength_cells=wavelength_cells))


def laser_ramp(n=(256, 128, 128), ppc=64, a0=3.0, wavelength_cells=16, waist_cells=24.0,
               duration_wavelengths=8, ramp=(128, 160), seed=1239, steps=500,
               name="laser_ramp") -> Workload:
    """Electrons filling x in [ramp[0], n_x) cells with a weight ramp 0 -> 1 n_crit
    over the `ramp` cells; a +x Gaussian-waisted pulse Ey = Bz = a0 sin(k(x - x0))
    env(x) exp(-r^2 / waist^2), env a sin^2 window of `duration_wavelengths`
    wavelengths from x = 0; absorbing in x, periodic in y and z."""
    rng = np.random.default_rng(seed)
    delta = 2.0 * math.pi / wavelength_cells
    d = (delta, delta, delta)
    cells = _cells_repeated(n, ppc, ((ramp[0], n[0]), (0, n[1]), (0, n[2])))
    npart = cells.shape[0]
    pos = (cells + rng.random((npart, 3))) * delta
    xr0, xr1 = ramp[0] * delta, ramp[1] * delta
    dens = np.clip((pos[:, 0] - xr0) / (xr1 - xr0), 0.0, 1.0)
    w = dens * delta ** 3 / ppc
    zero = np.zeros(npart)
    sp = Species(-1.0, 1.0, pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(), zero.copy(),
                 zero.copy(), zero.copy(), w)
    shape = (3, n[2], n[1], n[0])
    E = np.zeros(shape)
    B = np.zeros(shape)
    k = 2.0 * math.pi / (wavelength_cells * delta)
    x1 = duration_wavelengths * wavelength_cells * delta
    yc, zc = 0.5 * n[1] * delta, 0.5 * n[2] * delta
    w0 = waist_cells * delta

    def profile(x, y, z):
        env = np.where((x >= 0) & (x < x1), np.sin(math.pi * x / x1) ** 2, 0.0)
        r2 = (y - yc) ** 2 + (z - zc) ** 2
        return a0 * np.sin(k * x) * env * np.exp(-r2 / w0 ** 2)

    E[1] = profile(*_positions(n, d, 1, False))
    B[2] = profile(*_positions(n, d, 2, True))
    return Workload(name, tuple(n), d, courant_dt(d), steps, [sp], E, B,
                    bc=(ABSORBING, PERIODIC, PERIODIC),
                    meta=dict(ppc=ppc, a0=a0, seed=seed, ramp=ramp, waist_cells=waist_cells))


def config(name: str, seed: Optional[int] = None) -> Workload:
    """The named workloads.

    c1 -- 16^3 periodic, 8 e-/cell, vth 0.05c, 50 steps (parity size)
    c2 -- 64^3 periodic, 50 e-/cell (13.1 M), vth 0.05c, 1% density
          perturbation along x, 100 steps (paper-like scale; FP64 bench case)
    c3 -- 128^3 periodic, 32 e-/cell (67.1 M), vth 0.1c, 200 steps (mixed)
    c4 -- 32x32x64, slab z in [24,40) at 0.1 n_crit, 16 e-/cell, a0 = 1 plane
          wave, absorbing z, 200 steps (differentiable)
    c5 -- 256x128x128, 64 e-/cell over x in [128,256) with a 32-cell ramp
          (134.2 M), a0 = 3 Gaussian pulse, absorbing x, 500 steps
    r  -- 40^3 periodic, 50 e-/cell, vth 0.05c, 1000 steps (the paper's
          frozen-plasma size)
    """
    name = name.lower()
    if name == "c1":
        return uniform_plasma((16, 16, 16), 8, 0.05, 0.05, seed=1235 if seed is None else seed,
                              steps=50, name="c1")
    if name == "c2":
        return uniform_plasma((64, 64, 64), 50, 0.05, 0.05, seed=1236 if seed is None else seed,
                              perturb_eps=0.01, steps=100, name="c2")
    if name == "c3":
        return uniform_plasma((128, 128, 128), 32, 0.05, 0.1, seed=1237 if seed is None else seed,
                              steps=200, name="c3")
    if name == "c4":
        return laser_slab(seed=1238 if seed is None else seed)
    if name == "c5":
        return laser_ramp(seed=1239 if seed is None else seed)
    if name == "r":
        return uniform_plasma((40, 40, 40), 50, 0.05, 0.05, seed=1240 if seed is None else seed,
                              steps=1000, name="r")
    raise ValueError("unknown workload %r" % name)
