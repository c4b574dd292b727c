"""Parity at the benchmark's full sizes, in its launch configuration.

c2 (64^3 cells, 50 electrons per cell, 13,107,200 particles, FP64) and c3
(128^3, 32 per cell, 67,108,864 particles, mixed) are too large for the oracle
to step whole in a test, so one GPU step from a developed state (fields grown
by the plasma, particles drifted and re-sorted) is checked through:
* sampled particles, pushed one by one by the oracle from the same state
  (gather, Boris, move) -- positions and momenta element by element;
* the discrete charge continuity (rho^{n+1} - rho^n)/dt + div J = 0 of the
  GPU's current against CIC rho of all GPU particles (a property that holds
  at any size);
* the Yee update: the oracle's FDTD sub-steps applied to the GPU's E^n, B^n
  and the GPU's own J^{n+1/2} reproduce the GPU's E^{n+1}, B^{n+1}.
"""
import numpy as np
import pytest

import oracle as O
from paper_1608_01009_gb300 import pic as P
from paper_1608_01009_gb300 import workloads as W
from tests import parity as PT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _state(sim, wl):
    E, B = sim.get_fields()
    p = sim.get_particles(0)
    o = np.argsort(p["id"])
    return E, B, {k: v[o] for k, v in p.items()}


def _full_size_check(name, precision, warm, nsample, tol_particles, tol_fields, tol_cont):
    wl = W.config(name)
    sim = P.Simulation.from_workload(wl, precision=precision, supercell=4)
    sim.step(warm)
    E0, B0, p0 = _state(sim, wl)
    sim.step(1)
    sim.sync()
    E1, B1, p1 = _state(sim, wl)
    J = sim.get_current()
    sim.close()
    n = p0["x"].shape[0]
    assert np.array_equal(p0["id"], p1["id"]) and n == wl.nparticles
    sp = wl.species[0]
    L = np.array(wl.n) * np.array(wl.d)

    # sampled particles, pushed one by one by the oracle from the same state
    rng = np.random.default_rng(77)
    idx = np.sort(rng.choice(n, size=nsample, replace=False))
    osp = O.OracleSpecies(sp.q, sp.m, *[p0[k][idx] for k in ("x", "y", "z", "ux", "uy", "uz", "w")])
    ora = O.Oracle(wl.n, wl.d, wl.dt, wl.bc, wl.absorb_cells, wl.absorb_sigma, E0, B0, [osp])
    ora.push_deposit(osp)
    for a, k in enumerate(("x", "y", "z")):
        dx = (p1[k][idx] - osp.arr[a] + 0.5 * L[a]) % L[a] - 0.5 * L[a]
        assert np.max(np.abs(dx)) / L[a] <= tol_particles, (k, np.max(np.abs(dx)) / L[a])
    for a, k in enumerate(("ux", "uy", "uz")):
        e = PT.rel_err(p1[k][idx], osp.arr[3 + a])
        assert e <= tol_particles, (k, e)

    # charge continuity of the GPU current over every particle
    s0 = O.OracleSpecies(sp.q, sp.m, p0["x"], p0["y"], p0["z"], p0["ux"], p0["uy"], p0["uz"], p0["w"])
    s1 = O.OracleSpecies(sp.q, sp.m, p1["x"], p1["y"], p1["z"], p1["ux"], p1["uy"], p1["uz"], p1["w"])
    g = O.Oracle(wl.n, wl.d, wl.dt, species=[s0])
    r0 = g.rho()
    r1 = O.Oracle(wl.n, wl.d, wl.dt, species=[s1]).rho()
    divJ = g.div(J)
    resid = (r1 - r0) / wl.dt + divJ
    assert np.max(np.abs(resid)) <= tol_cont * np.max(np.abs(divJ))

    # the Yee update with the GPU's own current
    f = O.Oracle(wl.n, wl.d, wl.dt, wl.bc, wl.absorb_cells, wl.absorb_sigma, E0, B0)
    f.J[:] = J
    f.fdtd_b_half()
    f.fdtd_e()
    f.fdtd_b_half()
    assert PT.rel_err(E1, f.E) <= tol_fields
    assert PT.rel_err(B1, f.B) <= tol_fields


def test_c2_full_size_fp64():
    _full_size_check("c2", P.FP64, warm=7, nsample=200_000, tol_particles=1e-12, tol_fields=1e-12,
                     tol_cont=1e-11)


def test_c3_full_size_mixed():
    # FP32 state: positions/momenta at FP32 rounding against the FP64 oracle step
    # from the same (FP32-rounded) state; continuity and Yee are exact in FP64
    _full_size_check("c3", P.MIXED, warm=4, nsample=200_000, tol_particles=1e-6, tol_fields=1e-12,
                     tol_cont=1e-5)
