"""Hand-written adjoint (pic_tape_forward / pic_tape_backward) on the GPU.

Checks, in order of strength:
* transpose: the field-only adjoint is the exact transpose of the linear Yee
  map, <dL/dF0, v> = <g, F_N(v)> (dot-product test), periodic and absorbing;
* against the oracle's forward-mode tangent (the same plain FP64 CPU step run
  in dual numbers, independent of the CUDA path): the directional derivative
  of the final kinetic energy along random (E0, B0, x0, u0) directions;
* against central finite differences of the GPU forward (h = 1e-6, 1e-6 relative);
* checkpoint interval does not change the gradient, also where particles
  leave through an absorbing face between the recorded positions, and a
  second backward of the same tape gives the first one's gradient;
* the torch.autograd.Function and the gradient with respect to a laser
  amplitude a0 (through the linear initialiser).
"""
import numpy as np
import pytest

import oracle as O
from paper_1608_01009_gb300 import pic as P
from paper_1608_01009_gb300 import workloads as W
from tests import parity as PT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _vacuum_sim(n, bc, d=(0.05, 0.06, 0.045), absorb=4):
    dt = 0.5 / np.sqrt(sum(1 / x ** 2 for x in d))
    return P.Simulation(n, d, dt, bc=bc, absorb_cells=absorb, absorb_sigma=0.2)


@pytest.mark.parametrize("bc", [(0, 0, 0), (0, 0, 1), (1, 0, 1)])
def test_field_adjoint_is_the_transpose(bc):
    n = (8, 12, 16)
    rng = np.random.default_rng(31)
    shape = (3, n[2], n[1], n[0])
    vE, vB, gE, gB = (rng.standard_normal(shape) for _ in range(4))
    sim = _vacuum_sim(n, bc)
    sim.set_fields(vE, vB)
    sim.tape_forward(17, 5)
    EN, BN = sim.get_fields()
    lhs_forward = float(np.sum(gE * EN) + np.sum(gB * BN))
    dE0, dB0 = sim.tape_backward(0.0, _t(gE), _t(gB))
    rhs = float(np.sum(dE0.cpu().numpy() * vE) + np.sum(dB0.cpu().numpy() * vB))
    assert abs(lhs_forward - rhs) <= 1e-12 * max(abs(lhs_forward), 1.0)
    sim.close()


def _small_slab():
    return W.laser_slab(n=(8, 8, 32), ppc=2, slab=(10, 18), window=(2, 8), wavelength_cells=6, a0=1.5,
                        seed=41)


def _directions(wl, seed=5):
    rng = np.random.default_rng(seed)
    vE = rng.standard_normal(wl.E.shape)
    vB = rng.standard_normal(wl.B.shape)
    sp = wl.species[0]
    vx = [rng.standard_normal(sp.n) * d for d in wl.d]  # positions in physical units
    vu = [rng.standard_normal(sp.n) for _ in range(3)]
    return vE, vB, vx, vu


def _gpu_gradient(wl, nsteps, ckpt):
    sim = PT.make_sim(wl)
    wk = sim.tape_forward(nsteps, ckpt)
    dE0, dB0 = sim.tape_backward(1.0)
    dP = sim.tape_particle_grad(0)
    out = (wk, dE0.cpu().numpy(), dB0.cpu().numpy(), {k: v.cpu().numpy() for k, v in dP.items()})
    sim.close()
    return out


def _directional(dE0, dB0, dP, vE, vB, vx, vu):
    s = np.sum(dE0 * vE) + np.sum(dB0 * vB)
    for a, k in enumerate(("x", "y", "z")):
        s += np.sum(dP[k] * vx[a])
    for a, k in enumerate(("ux", "uy", "uz")):
        s += np.sum(dP[k] * vu[a])
    return float(s)


def test_adjoint_matches_oracle_tangent():
    wl = _small_slab()
    nsteps = 30
    wk, dE0, dB0, dP = _gpu_gradient(wl, nsteps, 7)
    vE, vB, vx, vu = _directions(wl)
    ora = O.Oracle.from_workload(wl)
    # step_tangent overwrites its tangent arrays with the final tangents: pass copies
    ptan = [[np.array(a, dtype=np.float64, copy=True) for a in (vx[0], vx[1], vx[2], vu[0], vu[1], vu[2])] +
            [np.zeros(wl.species[0].n)]]
    wk_o, dwk_o = ora.step_tangent(vE.copy(), vB.copy(), ptan, nsteps)
    assert abs(wk - wk_o) <= 1e-12 * abs(wk_o)
    got = _directional(dE0, dB0, dP, vE, vB, vx, vu)
    assert abs(got - dwk_o) <= 1e-9 * abs(dwk_o), (got, dwk_o)


def test_adjoint_matches_oracle_tangent_laser_ramp():
    # x absorbing, Gaussian pulse, weight ramp (config-5 features at small size)
    wl = W.laser_ramp(n=(32, 8, 8), ppc=2, a0=2.0, wavelength_cells=8, waist_cells=3.0, duration_wavelengths=2,
                      ramp=(16, 24), seed=19)
    nsteps = 40
    wk, dE0, dB0, dP = _gpu_gradient(wl, nsteps, 9)
    vE, vB, vx, vu = _directions(wl, seed=23)
    ora = O.Oracle.from_workload(wl)
    ptan = [[np.array(a, dtype=np.float64, copy=True) for a in (vx[0], vx[1], vx[2], vu[0], vu[1], vu[2])] +
            [np.zeros(wl.species[0].n)]]
    wk_o, dwk_o = ora.step_tangent(vE.copy(), vB.copy(), ptan, nsteps)
    assert abs(wk - wk_o) <= 1e-12 * abs(wk_o)
    got = _directional(dE0, dB0, dP, vE, vB, vx, vu)
    assert abs(got - dwk_o) <= 1e-9 * abs(dwk_o), (got, dwk_o)


def test_adjoint_matches_central_differences():
    wl = _small_slab()
    nsteps = 24
    wk, dE0, dB0, dP = _gpu_gradient(wl, nsteps, 6)
    vE, vB, _, _ = _directions(wl, seed=9)
    got = float(np.sum(dE0 * vE) + np.sum(dB0 * vB))

    def L(h):
        w = wl.copy()
        w.E = w.E + h * vE
        w.B = w.B + h * vB
        sim = PT.make_sim(w)
        v = sim.tape_forward(nsteps, nsteps)
        sim.close()
        return v

    # random perturbations of every field value make the third derivative large:
    # h = 1e-6 keeps the truncation error of the central difference near 1e-8
    h = 1e-6
    fd = (L(h) - L(-h)) / (2 * h)
    assert abs(fd - got) <= 1e-6 * abs(got), (fd, got)


def test_checkpoint_interval_does_not_change_gradient():
    wl = _small_slab()
    ref = _gpu_gradient(wl, 20, 20)
    for ck in (1, 3, 7):
        g = _gpu_gradient(wl, 20, ck)
        assert abs(g[0] - ref[0]) <= 1e-14 * abs(ref[0])
        assert np.max(np.abs(g[1] - ref[1])) <= 1e-12 * np.max(np.abs(ref[1]))
        assert np.max(np.abs(g[2] - ref[2])) <= 1e-12 * np.max(np.abs(ref[2]))


@pytest.mark.parametrize("ckpt", [20, 3, 7])
def test_repeated_backward_gives_the_same_gradient(ckpt):
    # a second backward of the same tape: with several segments the first one replayed
    # the early segments over the final state, which the second brings back before it
    # seeds the kinetic-energy cotangent
    wl = _small_slab()
    sim = PT.make_sim(wl)
    sim.tape_forward(20, ckpt)
    out = []
    for _ in range(2):
        dE0, dB0 = sim.tape_backward(1.0)
        dP = sim.tape_particle_grad(0)
        out.append((dE0.cpu().numpy(), dB0.cpu().numpy(), dP["ux"].cpu().numpy()))
    sim.close()
    for a in range(3):
        ref = out[0][a]
        assert np.max(np.abs(ref)) > 0.0
        assert np.max(np.abs(out[1][a] - ref)) <= 1e-12 * np.max(np.abs(ref)), a


def test_rebuilt_positions_follow_absorbing_exits():
    # a hot plasma in a box absorbing along z: particles leave during the recorded
    # segment, so the positions and active flags rebuilt between every 5th step of a
    # one-segment tape must follow the forward's own moves, exits included; a tape
    # with a checkpoint every step rebuilds nothing
    wl = W.uniform_plasma(n=(8, 8, 16), ppc=2, vth=0.6, seed=57)
    wl.bc, wl.absorb_cells, wl.absorb_sigma = (0, 0, 1), 3, 0.2
    nsteps = 25
    sim = PT.make_sim(wl)
    sim.tape_forward(nsteps, nsteps)
    left = sim.count()
    sim.close()
    assert 0 < left < wl.nparticles - 20, left
    ref = _gpu_gradient(wl, nsteps, 1)
    g = _gpu_gradient(wl, nsteps, nsteps)
    assert abs(g[0] - ref[0]) <= 1e-14 * abs(ref[0])
    for a in (1, 2):
        assert np.max(np.abs(g[a] - ref[a])) <= 1e-12 * np.max(np.abs(ref[a]))
    for k in ("x", "y", "z", "ux", "uy", "uz"):
        assert np.max(np.abs(g[3][k] - ref[3][k])) <= 1e-12 * np.max(np.abs(ref[3][k])), k


def test_tape_forward_matches_oracle_and_pic_step():
    wl = _small_slab()
    sim = PT.make_sim(wl)
    wk = sim.tape_forward(15, 4)
    ora = O.Oracle.from_workload(wl)
    ora.step(15)
    errs = dict(PT.field_errors(sim, ora))
    errs.update(PT.particle_errors(sim, ora, wl))
    # every array, the current J^{n+1/2} of the last tape step included
    assert max(errs.values()) <= 1e-11, errs
    assert abs(wk - ora.kinetic_energy()) <= 1e-12 * abs(wk)
    # and the context carries on with the fast path from the tape's final state
    sim.step(3)
    ora.step(3)
    errs = dict(PT.field_errors(sim, ora))
    errs.update(PT.particle_errors(sim, ora, wl))
    assert max(errs.values()) <= 1e-10, errs
    sim.close()


def test_autograd_function_and_a0_gradient():
    from paper_1608_01009_gb300.adjoint import kinetic_energy_after
    wl = _small_slab()
    a0_base = wl.meta["a0"]
    profE = _t(wl.E / a0_base)
    profB = _t(wl.B / a0_base)
    sp = wl.species[0]
    nsteps = 24

    def loss(a0):
        sim = PT.make_sim(wl)
        v = kinetic_energy_after(a0 * profE, a0 * profB, sim, nsteps, 8)
        return v, sim

    a0 = torch.tensor(a0_base, dtype=torch.float64, device="cuda", requires_grad=True)
    L, sim = loss(a0)
    L.backward()
    g = float(a0.grad.item())
    sim.close()
    with torch.no_grad():
        h = 1e-6
        vals = {}
        for s in (h, -h):
            v, sm = loss(torch.tensor(a0_base + s, dtype=torch.float64, device="cuda"))
            vals[s] = float(v.item())
            sm.close()
    fd = (vals[h] - vals[-h]) / (2 * h)
    assert abs(fd - g) <= 1e-6 * abs(g), (fd, g)
    assert g > 0  # a stronger pulse heats the slab more


def test_c4_a0_gradient_matches_central_differences():
    # at the size and schedule the benchmark times: the laser slab c4 (262,144
    # electrons), W_K after 200 steps, checkpoint every 20; dW_K/da0 through the
    # autograd Function against a central difference of two forward runs
    from paper_1608_01009_gb300.adjoint import kinetic_energy_after
    wl = W.config("c4")
    a0_base = wl.meta["a0"]
    profE = _t(wl.E / a0_base)
    profB = _t(wl.B / a0_base)

    def loss(a0):
        sim = PT.make_sim(wl)
        v = kinetic_energy_after(a0 * profE, a0 * profB, sim, 200, 20)
        return v, sim

    a0 = torch.tensor(a0_base, dtype=torch.float64, device="cuda", requires_grad=True)
    L, sim = loss(a0)
    L.backward()
    g = float(a0.grad.item())
    sim.close()
    h = 1e-6
    vals = {}
    with torch.no_grad():
        for s in (h, -h):
            v, sm = loss(torch.tensor(a0_base + s, dtype=torch.float64, device="cuda"))
            vals[s] = float(v.item())
            sm.close()
    fd = (vals[h] - vals[-h]) / (2 * h)
    rel = abs(fd - g) / abs(g)
    print("c4 dW_K/da0: adjoint %.15e, central difference %.15e, relative difference %.2e" % (g, fd, rel))
    assert rel <= 1e-6, (fd, g, rel)
