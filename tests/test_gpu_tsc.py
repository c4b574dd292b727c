"""Second-order (TSC) form factor with the Esirkepov current on the GPU
against the FP64 oracle (form_factor = 2), element by element.

Bar: the FP64 path's 1e-12 per step, norm-wise per array.  Cases: one step
from the workload's state and from a developed state (drift and sorts), a
hot plasma with multi-face moves, random initial fields, an absorbing laser
slab with particles leaving, several supercell sizes, ten-step
trajectories, two species, and the discrete charge continuity of the GPU's
own current against TSC rho at a size the oracle only samples; checkpoint
and resume of a TSC run, and blobs of the other form factor refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_1608_01009_gb300 import pic as P
from paper_1608_01009_gb300 import workloads as W
from tests import parity as PT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _sim(wl, supercell=4, sort_interval=0):
    return P.Simulation.from_workload(wl, supercell=supercell, sort_interval=sort_interval, form_factor=2)


def _oracle_from_gpu(sim, wl):
    ora = PT.oracle_from_gpu(sim, wl)
    ora.grid.form_factor = 2
    return ora


def _check(wl, steps=1, warm=0, supercell=4, tol=TOL):
    sim = _sim(wl, supercell)
    if warm:
        sim.step(warm)
        sim.sync()
    ora = _oracle_from_gpu(sim, wl)
    sim.step(steps)
    sim.sync()
    ora.step(steps)
    errs = dict(PT.field_errors(sim, ora))
    for s in range(len(wl.species)):
        for k, v in PT.particle_errors(sim, ora, wl, s).items():
            errs["p%d_%s" % (s, k)] = v
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad
    wf, wk = sim.energy()
    assert abs(wk - ora.kinetic_energy()) <= 1e-12 * abs(ora.kinetic_energy())
    sim.close()


def test_tsc_c1_first_step():
    _check(W.config("c1"))


def test_tsc_after_drift_and_sorts():
    _check(W.config("c1"), warm=7)


@pytest.mark.parametrize("S", [2, 4, 8])
def test_tsc_hot_plasma_supercells(S):
    _check(W.uniform_plasma((16, 8, 24), 6, 0.05, 0.3, seed=73), supercell=S, warm=2)


def test_tsc_non_cubic_cells():
    _check(W.uniform_plasma((12, 8, 16), 4, (0.05, 0.06, 0.045), 0.25, seed=80), warm=2)


def test_tsc_random_initial_fields():
    wl = W.uniform_plasma((12, 16, 8), 5, 0.05, 0.1, seed=74)
    rng = np.random.default_rng(75)
    wl.E = 0.5 * rng.standard_normal(wl.E.shape)
    wl.B = 0.5 * rng.standard_normal(wl.B.shape)
    _check(wl)


def test_tsc_absorbing_slab_with_laser():
    wl = W.laser_slab(n=(8, 8, 32), ppc=4, slab=(10, 18), window=(2, 8), wavelength_cells=6, a0=2.0, seed=76)
    _check(wl, warm=10)


def test_tsc_particles_leave_through_absorbing_faces():
    wl = W.uniform_plasma((8, 8, 16), 2, 0.05, 0.01, seed=79)
    wl.bc = (0, 0, 1)
    wl.absorb_cells = 2
    sp = wl.species[0]
    sp.uz[:] = np.where(sp.z < 0.4, -3.0, 3.0)
    sim = _sim(wl)
    sim.step(10)
    ora = _oracle_from_gpu(sim, wl)
    n_before = sim.count()
    sim.step(1)
    ora.step(1)
    errs = dict(PT.particle_errors(sim, ora, wl))
    errs.update(PT.field_errors(sim, ora))
    assert max(errs.values()) <= TOL, errs
    assert sim.count() < n_before
    sim.close()


def test_tsc_ten_step_trajectories():
    _check(W.uniform_plasma((8, 8, 12), 8, 0.05, 0.2, seed=77), steps=10, tol=1e-11)


def test_tsc_charge_continuity_at_size():
    wl = W.uniform_plasma((32, 32, 32), 20, 0.05, 0.1, seed=78)
    sim = _sim(wl)
    sim.step(3)
    p0 = sim.get_particles(0)
    sim.step(1)
    sim.sync()
    p1 = sim.get_particles(0)
    J = sim.get_current()
    sim.close()
    sp = wl.species[0]

    def rho(p):
        o = np.argsort(p["id"])
        s = O.OracleSpecies(sp.q, sp.m, *[p[k][o] for k in ("x", "y", "z", "ux", "uy", "uz", "w")])
        return O.Oracle(wl.n, wl.d, wl.dt, species=[s], form_factor=2).rho()

    g = O.Oracle(wl.n, wl.d, wl.dt, form_factor=2)
    divJ = g.div(J)
    resid = (rho(p1) - rho(p0)) / wl.dt + divJ
    assert np.max(np.abs(resid)) <= 1e-11 * np.max(np.abs(divJ))


def test_tsc_rejects_the_tape():
    sim = _sim(W.config("c1"))
    with pytest.raises(P.PicError) as ei:
        sim.tape_forward(2, 1)
    assert ei.value.code == -7  # PIC_ERR_STATE
    sim.close()


def _two_species():
    wl = W.uniform_plasma((12, 8, 16), 5, 0.05, 0.15, seed=91)
    pos = W.uniform_plasma((12, 8, 16), 3, 0.05, 0.1, seed=92, q=1.0, m=1.0)
    wl.species = wl.species + pos.species
    return wl


def test_tsc_two_species():
    # electrons and positrons: both deposit into the same current, one oracle step
    _check(_two_species(), warm=4)


def test_tsc_checkpoint_resume_and_form_factor_mismatch():
    wl = _two_species()
    a = _sim(wl)
    a.step(4)
    blob = a.get_state()
    a.step(5)
    b = _sim(W.uniform_plasma((12, 8, 16), 1, 0.05, 0.0, seed=1))  # other particles
    b.set_state(blob)
    b.step(5)
    for x, y in zip(a.get_fields() + (a.get_current(),), b.get_fields() + (b.get_current(),)):
        assert PT.rel_err(y, x) <= 1e-12
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
        assert np.array_equal(pa["id"][oa], pb["id"][ob])
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            assert PT.rel_err(pb[k][ob], pa[k][oa]) <= 1e-12, (s, k)
    # a blob of the CIC form factor does not load into a TSC context, nor the reverse
    cic = PT.make_sim(wl)
    with pytest.raises(P.PicError) as ei:
        cic.set_state(blob)
    assert ei.value.code == -1
    with pytest.raises(P.PicError) as ei:
        b.set_state(cic.get_state())
    assert ei.value.code == -1
    b.step(1)
    b.sync()
    for s in (a, b, cic):
        s.close()
