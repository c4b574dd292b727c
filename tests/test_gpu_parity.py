"""GPU FP64 path vs the FP64 oracle, element by element, through the C ABI.

Bar (from the method's FP64 statement): every field, current and particle
array within 1e-12 norm-wise relative error per step.  One-step parity is
checked from identical states (the workload's, and a GPU state after several
steps, sorts and supercell drift), at sizes the oracle finishes in seconds
that span several supercells, a ragged tail and the edge cases.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1608_01009_gb300 import workloads as W
from tests import parity as PT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _check_one_step(wl, supercell=4, sort_interval=0, warm_steps=0, tol=TOL):
    sim = PT.make_sim(wl, supercell=supercell, sort_interval=sort_interval)
    if warm_steps:
        sim.step(warm_steps)
        sim.sync()
    ora = PT.oracle_from_gpu(sim, wl)
    sim.step(1)
    sim.sync()
    ora.step(1)
    fe = PT.field_errors(sim, ora)
    errs = dict(fe)
    for s in range(len(wl.species)):
        for k, v in PT.particle_errors(sim, ora, wl, s).items():
            errs["p%d_%s" % (s, k)] = v
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "errors above %g: %s" % (tol, bad)
    sim.close()
    return errs


def _plasma(n=(16, 16, 16), ppc=8, vth=0.05, seed=11, **kw):
    return W.uniform_plasma(n, ppc, 0.05, vth, seed=seed, **kw)


def test_c1_first_step():
    _check_one_step(W.config("c1"))


def test_c1_after_drift_and_sorts():
    # state after 7 steps: 2 sorts (K = 3) and particles drifted inside their slack
    _check_one_step(W.config("c1"), warm_steps=7, sort_interval=3)


@pytest.mark.parametrize("S", [2, 4, 8])
def test_supercell_sizes(S):
    _check_one_step(_plasma((16, 8, 24), 6, vth=0.2, seed=3), supercell=S, warm_steps=2)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_sort_intervals(K):
    _check_one_step(_plasma((8, 12, 8), 5, vth=0.3, seed=4), sort_interval=K, warm_steps=4)


@pytest.mark.parametrize("S", [2, 4, 8])
def test_non_cubic_cells(S):
    # unequal cell sizes take the kernel's general (non-cubic) instantiation
    wl = W.uniform_plasma((16, 8, 24), 5, (0.05, 0.06, 0.045), 0.25, seed=18)
    rng = np.random.default_rng(19)
    wl.E = 0.3 * rng.standard_normal(wl.E.shape)
    wl.B = 0.3 * rng.standard_normal(wl.B.shape)
    _check_one_step(wl, supercell=S, warm_steps=3)


@pytest.mark.parametrize("S", [4, 8])
def test_largest_axis_extent(S):
    # 1024 cells along x: the largest index the packed 10-bit cell coordinate holds
    _check_one_step(_plasma((1024, 8, 8), 1, vth=0.3, seed=20), supercell=S, warm_steps=2)


def test_single_relativistic_particle():
    # one particle at gamma ~ 10 moving diagonally: crosses up to three faces per step
    wl = _plasma((8, 8, 8), 1, vth=0.0, seed=21)
    sp = wl.species[0]
    keep = np.array([123])
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        setattr(sp, k, np.ascontiguousarray(getattr(sp, k)[keep]))
    sp.ux[:] = 6.0
    sp.uy[:] = -5.0
    sp.uz[:] = 5.5
    rng = np.random.default_rng(22)
    wl.E = 0.2 * rng.standard_normal(wl.E.shape)
    wl.B = 0.2 * rng.standard_normal(wl.B.shape)
    _check_one_step(wl, warm_steps=5)


def test_hot_plasma_many_crossings():
    # vth = 0.5c: a large share of particles crosses 1-3 cell faces per step
    _check_one_step(_plasma((8, 8, 8), 10, vth=0.5, seed=5), warm_steps=3)


def test_fields_and_particles_with_initial_fields():
    wl = _plasma((12, 8, 8), 4, vth=0.1, seed=6)
    rng = np.random.default_rng(6)
    wl.E[:] = 0.3 * rng.standard_normal(wl.E.shape)
    wl.B[:] = 0.3 * rng.standard_normal(wl.B.shape)
    _check_one_step(wl)
    _check_one_step(wl, warm_steps=5)


def test_perturbed_plasma_c2_shape_small():
    _check_one_step(W.uniform_plasma((16, 16, 16), 50, 0.05, 0.05, seed=7, perturb_eps=0.01), warm_steps=2)


def test_dense_bins_split_into_chunks():
    # > 4096 particles per supercell: each bin is cut into several chunks
    _check_one_step(_plasma((8, 8, 8), 80, vth=0.1, seed=8), warm_steps=1)


def test_ragged_occupancy_and_empty_bins():
    # particles only in a corner region: most supercells are empty
    wl = _plasma((16, 16, 16), 3, vth=0.2, seed=9)
    sp = wl.species[0]
    keep = (sp.x < 0.3) & (sp.y < 0.45) & (sp.z > 0.2)
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        setattr(sp, k, getattr(sp, k)[keep].copy())
    _check_one_step(wl, warm_steps=2)


def test_particles_on_faces_and_box_edge():
    # positions exactly on cell faces, on the box's lower edge, and just below its upper edge
    wl = _plasma((8, 8, 8), 1, vth=0.2, seed=10)
    sp = wl.species[0]
    L = 8 * 0.05
    sp.x[:64] = np.round(sp.x[:64] / 0.05) * 0.05
    sp.y[64:128] = 0.0
    sp.z[128:192] = np.nextafter(L, 0)
    _check_one_step(wl)


def test_zero_weight_and_two_species():
    wl = _plasma((8, 8, 16), 4, vth=0.2, seed=12)
    e = wl.species[0]
    e.w[::5] = 0.0
    pos = W.uniform_plasma((8, 8, 16), 2, 0.05, 0.1, seed=13).species[0]
    pos.q, pos.m = 1.0, 1836.0
    wl.species.append(pos)
    _check_one_step(wl, warm_steps=2)


def test_empty_species():
    wl = _plasma((8, 8, 8), 1, vth=0.1, seed=14)
    sp = wl.species[0]
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        setattr(sp, k, getattr(sp, k)[:0].copy())
    rng = np.random.default_rng(14)
    wl.E[:] = rng.standard_normal(wl.E.shape)
    errs = _check_one_step(wl, warm_steps=2)
    assert errs["Jx"] == 0.0


def test_absorbing_slab_with_laser():
    wl = W.laser_slab(n=(8, 8, 32), ppc=4, slab=(10, 18), window=(2, 8), wavelength_cells=6, a0=2.0)
    _check_one_step(wl, warm_steps=10)


def test_absorbing_particles_leave():
    # particles streaming out through the absorbing z faces are deactivated identically
    wl = _plasma((8, 8, 16), 2, vth=0.01, seed=15)
    wl.bc = (0, 0, 1)
    wl.absorb_cells = 2
    sp = wl.species[0]
    sp.uz[:] = np.where(sp.z < 0.4, -3.0, 3.0)
    sim = PT.make_sim(wl)
    sim.step(10)
    ora = PT.oracle_from_gpu(sim, wl)
    n_before = sim.count()
    sim.step(1)
    ora.step(1)
    errs = PT.particle_errors(sim, ora, wl)
    assert max(errs.values()) <= TOL
    assert sim.count() < n_before
    fe = PT.field_errors(sim, ora)
    assert max(fe.values()) <= TOL, fe


def test_every_particle_leaves():
    # absorbing z, every particle streaming out: the store empties through the
    # sort's compaction and the empty species keeps stepping
    wl = _plasma((8, 8, 8), 2, vth=0.01, seed=23)
    wl.bc = (0, 0, 1)
    wl.absorb_cells = 2
    sp = wl.species[0]
    sp.uz[:] = np.where(sp.z < 0.2, -4.0, 4.0)
    sim = PT.make_sim(wl)
    ora = O.Oracle.from_workload(wl)
    sim.step(40)
    ora.step(40)
    sim.sync()
    assert sim.count() == 0 and int(ora.species[0].active.sum()) == 0
    errs = PT.field_errors(sim, ora)
    assert max(errs.values()) <= 1e-11, errs
    sim.close()


def test_multi_step_trajectory_c1():
    # five whole steps from the workload state: errors stay at rounding level
    wl = W.config("c1")
    sim = PT.make_sim(wl)
    ora = PT.oracle_from_gpu(sim, wl)
    sim.step(5)
    ora.step(5)
    errs = dict(PT.field_errors(sim, ora), **PT.particle_errors(sim, ora, wl))
    assert max(errs.values()) <= 1e-11, errs


def test_energy_diagnostics_match_oracle():
    wl = W.config("c1")
    sim = PT.make_sim(wl)
    sim.step(4)
    ora = PT.oracle_from_gpu(sim, wl)
    wf, wk = sim.energy()
    assert abs(wf - ora.field_energy()) <= 1e-12 * abs(ora.field_energy())
    assert abs(wk - ora.kinetic_energy()) <= 1e-12 * abs(ora.kinetic_energy())


def test_status_and_launch_count():
    wl = W.config("c1")
    sim = PT.make_sim(wl, sort_interval=3)
    sim.launch_count(reset=True)
    sim.step(6)
    sim.sync()
    # per step: 1 push + 3 field + 1 energy; one sort (5 kernels) at the 4th step (K = 3)
    assert sim.launch_count() == 6 * 5 + 5
    sim.close()
    # the FP64 default sorts before every step after the first (the load sorted)
    sim = PT.make_sim(wl)
    sim.launch_count(reset=True)
    sim.step(6)
    sim.sync()
    assert sim.launch_count() == 6 * 5 + 5 * 5
    sim.close()


def test_non_finite_input_is_reported_not_trapped():
    wl = _plasma((8, 8, 8), 2, vth=0.1, seed=16)
    sim = PT.make_sim(wl)
    E = np.array(wl.E)
    E[0, 3, 3, 3] = np.nan
    sim.set_fields(E, wl.B)
    sim.step(2)
    from paper_1608_01009_gb300 import pic as P
    with pytest.raises(P.PicError) as ei:
        sim.energy()
    assert ei.value.code == -5  # PIC_ERR_NAN
    sim.close()


def test_laser_ramp_small():
    # config-5 features at small size: x absorbing, Gaussian transverse pulse,
    # density ramp through the weights (weights from ~0 at the ramp foot)
    wl = W.laser_ramp(n=(32, 16, 16), ppc=2, a0=3.0, wavelength_cells=8, waist_cells=4.0,
                      duration_wavelengths=2, ramp=(16, 24), seed=17)
    _check_one_step(wl, warm_steps=12)
