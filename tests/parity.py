"""Helpers of the GPU-vs-oracle parity tests.

Metric (norm-wise relative error, per array): max|A_gpu - A_oracle| /
max(max|A_oracle|, tiny).  Particles are matched by id; positions compare
modulo the box on periodic axes.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1608_01009_gb300 import pic as P

TINY = 1e-300


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.size == 0 and b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), TINY))


def oracle_from_gpu(sim, wl):
    """Oracle state equal to the GPU's current state (fields + particles by id)."""
    E, B = sim.get_fields()
    species = []
    for s, sp in enumerate(wl.species):
        p = sim.get_particles(s)
        order = np.argsort(p["id"])
        osp = O.OracleSpecies(sp.q, sp.m, *[p[k][order] for k in ("x", "y", "z", "ux", "uy", "uz", "w")])
        osp.ids = p["id"][order]
        species.append(osp)
    ora = O.Oracle(wl.n, wl.d, wl.dt, wl.bc, wl.absorb_cells, wl.absorb_sigma, E, B, species)
    return ora


def particle_errors(sim, ora, wl, species=0):
    """Relative errors of positions and momenta of the active particles, the
    two active-id sets being equal (else AssertionError)."""
    p = sim.get_particles(species)
    osp = ora.species[species]
    act = osp.active.astype(bool)
    ids = getattr(osp, "ids", np.arange(osp.n))[act]
    gid = np.sort(p["id"])
    assert gid.shape == ids.shape and np.array_equal(gid, ids), "active particle sets differ"
    order = np.argsort(p["id"])
    L = np.array(wl.n) * np.array(wl.d)
    errs = {}
    for a, k in enumerate(("x", "y", "z")):
        g = p[k][order]
        o = osp.arr[a][act]
        diff = g - o
        if wl.bc[a] == 0:
            diff = (diff + 0.5 * L[a]) % L[a] - 0.5 * L[a]
        errs[k] = float(np.max(np.abs(diff)) / L[a]) if diff.size else 0.0
    for a, k in enumerate(("ux", "uy", "uz")):
        errs[k] = rel_err(p[k][order], osp.arr[3 + a][act])
    errs["w"] = rel_err(p["w"][order], osp.w[act])
    return errs


def field_errors(sim, ora):
    E, B = sim.get_fields()
    J = sim.get_current()
    errs = {}
    for c, k in enumerate("xyz"):
        errs["E" + k] = rel_err(E[c], ora.E[c])
        errs["B" + k] = rel_err(B[c], ora.B[c])
        errs["J" + k] = rel_err(J[c], ora.J[c])
    return errs


def make_sim(wl, precision=P.FP64, supercell=4, sort_interval=0):
    return P.Simulation.from_workload(wl, precision=precision, supercell=supercell, sort_interval=sort_interval)
