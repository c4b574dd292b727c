"""Parity at the benchmark's full sizes, in its launch configuration.

c2 (64^3 cells, 50 electrons per cell, 13,107,200 particles, FP64; with the
CIC and with the second-order TSC + Esirkepov form factor), c3 (128^3, 32 per
cell, 67,108,864 particles, mixed) and c5 (256x128x128, 64 per cell over the
back half, 134,217,728 particles, mixed, absorbing in x, a0 = 3 pulse) are too
large for the oracle to step whole in a test, so one GPU step from a developed
state (fields grown by the plasma or the pulse inside the plasma, particles
drifted and re-sorted) is checked through:
* sampled particles, pushed one by one by the oracle from the same state
  (gather, Boris, move) -- positions and momenta element by element;
* the whole current J^{n+1/2}, element by element, against the oracle's
  deposit of every particle from the same state (pushed in chunks; c2 and c3);
* the discrete charge continuity (rho^{n+1} - rho^n)/dt + div J = 0 of the
  GPU's current against the CIC (or TSC) rho of all GPU particles (a property that holds
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


KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")
CHUNK = 1 << 24  # particles per oracle call when summing rho over a whole state


def _sampled(p, ids):
    """The records of the given ids (ids are 0..n-1: an inverse permutation, not a sort)."""
    i = p["id"]
    assert i.min() >= 0 and i.max() < i.shape[0]
    where = np.empty_like(i)
    where[i] = np.arange(i.shape[0])
    assert np.array_equal(i[where[ids]], ids)
    return [p[k][where[ids]] for k in KEYS]


def _full_size_check(name, precision, warm, nsample, tol_x, tol_u, tol_fields, tol_cont, form_factor=1,
                     tol_J=None):
    wl = W.config(name)
    sim = P.Simulation.from_workload(wl, precision=precision, supercell=4, form_factor=form_factor)
    n, q, m = wl.nparticles, wl.species[0].q, wl.species[0].m
    wl.species = []  # the host copy of the particles is not needed any more
    L = np.array(wl.n) * np.array(wl.d)
    grid = (wl.n, wl.d, wl.dt, wl.bc, wl.absorb_cells, wl.absorb_sigma)
    kw = dict(form_factor=form_factor)

    def rho(p):
        r = np.zeros((wl.n[2], wl.n[1], wl.n[0]))
        for a in range(0, p["x"].shape[0], CHUNK):
            s_ = O.OracleSpecies(q, m, *[p[k][a:a + CHUNK] for k in KEYS])
            r += O.Oracle(*grid, species=[s_], **kw).rho()
        return r

    ids = np.sort(np.random.default_rng(77).choice(n, size=nsample, replace=False))
    sim.step(warm)
    E0, B0 = sim.get_fields()
    p = sim.get_particles(0)
    # no particle has left (the plasma sits away from absorbing faces for these steps)
    assert p["x"].shape[0] == n
    s0 = _sampled(p, ids)
    r0 = rho(p)
    Jo = None
    if tol_J is not None:
        # the oracle's current of every particle from this state (gather, push, move,
        # deposit), summed over chunks into one grid
        ora = O.Oracle(*grid, E0, B0, **kw)
        for a in range(0, p["x"].shape[0], CHUNK):
            ora.push_deposit(O.OracleSpecies(q, m, *[p[k][a:a + CHUNK] for k in KEYS]))
        Jo = ora.J
        del ora
    del p
    sim.step(1)
    sim.sync()
    E1, B1 = sim.get_fields()
    J = sim.get_current()
    p = sim.get_particles(0)
    assert p["x"].shape[0] == n
    s1 = _sampled(p, ids)
    r1 = rho(p)
    del p
    sim.close()

    # sampled particles, pushed one by one by the oracle from the same state
    osp = O.OracleSpecies(q, m, *s0)
    O.Oracle(*grid, E0, B0, [osp], **kw).push_deposit(osp)
    for a, k in enumerate(("x", "y", "z")):
        dx = (s1[a] - osp.arr[a] + 0.5 * L[a]) % L[a] - 0.5 * L[a]
        assert np.max(np.abs(dx)) / L[a] <= tol_x, (k, np.max(np.abs(dx)) / L[a])
    for a, k in enumerate(("ux", "uy", "uz")):
        e = PT.rel_err(s1[3 + a], osp.arr[3 + a])
        assert e <= tol_u, (k, e)

    # the whole current, element by element (norm-wise per component array)
    if Jo is not None:
        e = PT.rel_err(J, Jo)
        assert e <= tol_J, ("J", e)

    # charge continuity of the GPU current over every particle
    divJ = O.Oracle(*grid, **kw).div(J)
    assert np.max(np.abs(divJ)) > 0
    resid = (r1 - r0) / wl.dt + divJ
    assert np.max(np.abs(resid)) <= tol_cont * np.max(np.abs(divJ))

    # the Yee update with the GPU's own current
    f = O.Oracle(*grid, E0, B0)
    f.J[:] = J
    f.fdtd_b_half()
    f.fdtd_e()
    f.fdtd_b_half()
    assert PT.rel_err(E1, f.E) <= tol_fields
    assert PT.rel_err(B1, f.B) <= tol_fields


def test_c2_full_size_fp64():
    _full_size_check("c2", P.FP64, warm=7, nsample=200_000, tol_x=1e-12, tol_u=1e-12, tol_fields=1e-12,
                     tol_cont=1e-11, tol_J=1e-12)


def test_c2_full_size_tsc():
    # second-order form factor: TSC gather, Esirkepov current, continuity against TSC rho
    _full_size_check("c2", P.FP64, warm=7, nsample=100_000, tol_x=1e-12, tol_u=1e-12, tol_fields=1e-12,
                     tol_cont=1e-11, form_factor=2)


def test_c3_full_size_mixed():
    # FP32 state: positions/momenta at FP32 rounding against the FP64 oracle step
    # from the same (FP32-rounded) state; continuity and Yee are exact in FP64
    # J: FP32 gather, push and current sums against the FP64 oracle from the same state
    _full_size_check("c3", P.MIXED, warm=4, nsample=200_000, tol_x=1e-6, tol_u=1e-6, tol_fields=1e-12,
                     tol_cont=1e-5, tol_J=1e-5)


def test_c5_full_size_mixed_laser_ramp():
    # after 150 steps the pulse front is about 40 cells into the ramp: relativistic
    # electrons (a0 = 3), the absorbing layer, and a cold plasma elsewhere
    _full_size_check("c5", P.MIXED, warm=150, nsample=200_000, tol_x=1e-6, tol_u=1e-5, tol_fields=1e-12,
                     tol_cont=1e-5)
