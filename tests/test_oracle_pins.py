"""Pins of the FP64 CPU oracle against closed forms, invariants and brute force.

The oracle (oracle/pic_oracle.cpp) is what the CUDA path is compared with, so
it is itself checked here against results the method and the mathematics fix
(no GPU needed):

* gather    -- exact for uniform and for linear fields (CIC reproduces linear
               functions); equal to a direct sum of the hat function;
* Boris     -- |u| invariant in a pure B field; rotation angle 2 atan(|q|B dt/2m gamma);
               discrete orbit radius dt|u_perp| / (2 gamma sin(theta/2));
               equal to Rodrigues' rotation; E x B drift velocity;
* deposit   -- discrete charge continuity (rho^{n+1}-rho^n)/dt + div J = 0 for
               CIC rho; equal to the Gauss-Legendre line integral;
* FDTD      -- an exact discrete plane-wave eigenmode of the Yee scheme;
               the discrete vacuum energy invariant;
* whole step-- constancy of the Gauss-law residual div E - rho; a brute-force
               step-by-step restatement on a few particles;
* absorbing -- the damping factor at every staggered lattice point of the layer;
               a pulse entering the damping layer loses its energy; particles
               leaving the domain are deactivated.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests import bruteforce as bf

RNG = np.random.default_rng(20160803)


def _rand_fields(n, scale=1.0, rng=RNG):
    shape = (3, n[2], n[1], n[0])
    return scale * rng.standard_normal(shape), scale * rng.standard_normal(shape)


# ---------------------------------------------------------------- gather
def test_gather_uniform_field_exact():
    n, d = (5, 6, 7), (0.1, 0.2, 0.15)
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    ev, bv = (0.3, -1.7, 2.5), (-0.9, 0.4, 1.1)
    for c in range(3):
        E[c] = ev[c]
        B[c] = bv[c]
    ora = O.Oracle(n, d, 0.01, E=E, B=B)
    pos = RNG.random((200, 3)) * np.array(n) * np.array(d)
    Eo, Bo = ora.gather(pos[:, 0], pos[:, 1], pos[:, 2])
    for c in range(3):
        assert np.max(np.abs(Eo[c] - ev[c])) < 1e-15
        assert np.max(np.abs(Bo[c] - bv[c])) < 1e-15


def test_gather_linear_field_exact():
    # A linear field is reproduced exactly by CIC at positions whose 8 lattice
    # neighbours are inside the domain (absorbing axes, so no wrap).
    n, d = (8, 9, 10), (0.1, 0.07, 0.13)
    coef = RNG.standard_normal((6, 4))
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    zz, yy, xx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for c in range(3):
        for F, st, row in ((E, bf.STAG_E, c), (B, bf.STAG_B, 3 + c)):
            a0, a1, a2, a3 = coef[row]
            F[c] = a0 + a1 * (xx + st[c][0]) + a2 * (yy + st[c][1]) + a3 * (zz + st[c][2])
    ora = O.Oracle(n, d, 0.01, bc=(1, 1, 1), absorb_cells=0, E=E, B=B)
    xi = 1.0 + RNG.random((300, 3)) * (np.array(n) - 3)
    pos = xi * np.array(d)
    Eo, Bo = ora.gather(pos[:, 0], pos[:, 1], pos[:, 2])
    for c in range(3):
        for got, row in ((Eo[c], c), (Bo[c], 3 + c)):
            a0, a1, a2, a3 = coef[row]
            want = a0 + a1 * xi[:, 0] + a2 * xi[:, 1] + a3 * xi[:, 2]
            assert np.max(np.abs(got - want)) < 1e-13


def test_gather_matches_direct_hat_sum():
    n, d = (4, 5, 3), (0.05, 0.07, 0.04)
    E, B = _rand_fields(n)
    ora = O.Oracle(n, d, 0.01, E=E, B=B)
    pos = RNG.random((40, 3)) * np.array(n) * np.array(d)
    Eo, Bo = ora.gather(pos[:, 0], pos[:, 1], pos[:, 2])
    Eb, Bb = bf.gather(E, B, n, d, pos)
    assert np.max(np.abs(Eo.T - Eb)) < 1e-13
    assert np.max(np.abs(Bo.T - Bb)) < 1e-13


# ---------------------------------------------------------------- Boris
def _boris(u, E, B, q=-1.0, m=1.0, dt=0.01):
    u = np.array(np.asarray(u, dtype=np.float64).T, order="C", copy=True)
    n = u.shape[1]
    Ep = np.ascontiguousarray(np.broadcast_to(np.asarray(E, np.float64).reshape(3, -1), (3, n)))
    Bp = np.ascontiguousarray(np.broadcast_to(np.asarray(B, np.float64).reshape(3, -1), (3, n)))
    O.lib().or_boris(n, O._p(u), O._p(Ep), O._p(Bp), q, m, dt)
    return u.T


def test_boris_rotation_angle_and_invariance():
    # E = 0, B along z: |u| is invariant and u_perp turns by 2 atan(|q| B dt / (2 m gamma)).
    Bz, dt = 3.0, 0.05
    u0 = np.array([[0.3, 0.1, 0.2]])
    gam = math.sqrt(1 + u0[0] @ u0[0])
    theta = 2 * math.atan(Bz * dt / (2 * gam))
    u = u0.copy()
    for k in range(1, 101):
        u = _boris(u, (0, 0, 0), (0, 0, Bz), q=-1.0, dt=dt)
        assert abs(math.sqrt(u[0] @ u[0]) - math.sqrt(u0[0] @ u0[0])) < 2e-15
        ang = math.atan2(u[0, 1], u[0, 0]) - math.atan2(u0[0, 1], u0[0, 0])
        # an electron (q < 0) turns counter-clockwise about +B
        want = (k * theta + math.pi) % (2 * math.pi) - math.pi
        got = (ang + math.pi) % (2 * math.pi) - math.pi
        assert abs(((got - want) + math.pi) % (2 * math.pi) - math.pi) < 1e-12
        assert u[0, 2] == u0[0, 2]


def test_boris_matches_rodrigues_rotation():
    for _ in range(50):
        u = RNG.standard_normal(3) * 0.5
        E = RNG.standard_normal(3)
        B = RNG.standard_normal(3) * 4
        q, m, dt = RNG.choice([-1.0, 1.0]), RNG.uniform(0.5, 2.0), 0.03
        got = _boris(u[None, :], E, B, q=q, m=m, dt=dt)[0]
        want = bf.boris_rodrigues(u, E, B, q, m, dt)
        assert np.max(np.abs(got - want)) < 1e-14


def _single_particle_run(E0, B0, u0, x0, nsteps, dt=0.02, n=(8, 8, 8), delta=1.0):
    # zero weight: no current, so the uniform external fields stay static
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    for c in range(3):
        E[c] = E0[c]
        B[c] = B0[c]
    sp = O.OracleSpecies(-1.0, 1.0, [x0[0]], [x0[1]], [x0[2]], [u0[0]], [u0[1]], [u0[2]], [0.0])
    ora = O.Oracle(n, (delta,) * 3, dt, E=E, B=B, species=[sp])
    L = np.array(n) * delta
    xs, us = [np.array(x0, float)], [np.array(u0, float)]
    for _ in range(nsteps):
        ora.step(1)
        x = np.array([sp.x[0], sp.y[0], sp.z[0]])
        # unwrap across the periodic box
        prev = xs[-1]
        x = x + L * np.round((prev - x) / L)
        xs.append(x)
        us.append(np.array([sp.ux[0], sp.uy[0], sp.uz[0]]))
    return np.array(xs), np.array(us), ora


def test_gyration_radius_and_frequency():
    Bz, dt, u0 = 2.0, 0.02, np.array([0.4, 0.0, 0.0])
    gam = math.sqrt(1 + u0 @ u0)
    theta = 2 * math.atan(Bz * dt / (2 * gam))
    R = dt * 0.4 / (2 * gam * math.sin(theta / 2))
    xs, us, _ = _single_particle_run((0, 0, 0), (0, 0, Bz), u0, (4.0, 4.0, 4.0), 400, dt=dt)
    # circumcentre of the first three positions (plane z = const)
    a, b, c = xs[0, :2], xs[1, :2], xs[2, :2]
    D = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux_ = ((a @ a) * (b[1] - c[1]) + (b @ b) * (c[1] - a[1]) + (c @ c) * (a[1] - b[1])) / D
    uy_ = ((a @ a) * (c[0] - b[0]) + (b @ b) * (a[0] - c[0]) + (c @ c) * (b[0] - a[0])) / D
    r = np.hypot(xs[:, 0] - ux_, xs[:, 1] - uy_)
    assert np.max(np.abs(r - R)) < 1e-11 * max(1.0, R)
    # continuum limit: R -> r_L = |u_perp| / (|q| B)
    assert abs(R - 0.4 / Bz) / (0.4 / Bz) < 1e-3
    # frequency: the momentum turns by theta each step
    ang = np.unwrap(np.arctan2(us[:, 1], us[:, 0]))
    assert np.max(np.abs(ang - ang[0] - theta * np.arange(len(ang)))) < 1e-10


def test_exb_drift():
    # From rest in crossed uniform fields, averaged over whole gyro-periods the
    # guiding centre drifts at E x B / B^2 (relativistic corrections O(v_d^2)).
    B0 = np.array([0.0, 0.0, 5.0])
    E0 = np.array([0.05, 0.0, 0.0])
    vd = np.cross(E0, B0) / (B0 @ B0)
    dt = 0.01
    theta = 2 * math.atan(5.0 * dt / 2)
    period = 2 * math.pi / theta
    nper = 50
    nsteps = int(round(nper * period))
    xs, _, _ = _single_particle_run(E0, B0, (0, 0, 0), (4.0, 4.0, 4.0), nsteps, dt=dt)
    v = (xs[-1] - xs[0]) / (nsteps * dt)
    assert np.max(np.abs(v - vd)) / np.linalg.norm(vd) < 5e-3


# ---------------------------------------------------------------- deposit
def _random_moves(n, d, npart, maxstep, rng=RNG):
    L = np.array(n) * np.array(d)
    x0 = rng.random((npart, 3)) * L
    step = (rng.random((npart, 3)) * 2 - 1) * maxstep * np.array(d)
    return x0, x0 + step


def test_deposit_charge_continuity():
    n, d, dt, q = (6, 5, 7), (0.05, 0.04, 0.06), 0.013, -1.0
    x0, x1 = _random_moves(n, d, 300, 0.95)
    w = RNG.random(300) + 0.5
    ora = O.Oracle(n, d, dt)
    ora.deposit(x0.T, x1.T, w, q)
    L = np.array(n) * np.array(d)
    s0 = O.OracleSpecies(q, 1.0, x0[:, 0], x0[:, 1], x0[:, 2], *np.zeros((3, 300)), w)
    x1w = np.mod(x1, L)
    s1 = O.OracleSpecies(q, 1.0, x1w[:, 0], x1w[:, 1], x1w[:, 2], *np.zeros((3, 300)), w)
    r0 = O.Oracle(n, d, dt, species=[s0]).rho()
    r1 = O.Oracle(n, d, dt, species=[s1]).rho()
    divJ = ora.div(ora.J)
    resid = (r1 - r0) / dt + divJ
    assert np.max(np.abs(resid)) < 1e-13 * np.max(np.abs(divJ))


def test_deposit_matches_line_integral():
    n, d, dt, q = (5, 4, 6), (0.05, 0.07, 0.04), 0.011, 1.3
    x0, x1 = _random_moves(n, d, 40, 0.9)
    w = RNG.random(40) + 0.5
    ora = O.Oracle(n, d, dt)
    ora.deposit(x0.T, x1.T, w, q)
    J = np.zeros_like(ora.J)
    bf.deposit(J, n, d, dt, x0, x1, w, q)
    assert np.max(np.abs(ora.J - J)) < 1e-12 * np.max(np.abs(J))


def test_deposit_single_cell_special_case():
    # A move parallel to x inside one cell at transverse offsets (fy, fz):
    # Jx on the four x-edges is Q dx times the bilinear weights, nothing else.
    n, d, dt = (4, 4, 4), (1.0, 1.0, 1.0), 1.0
    ora = O.Oracle(n, d, dt)
    x0 = np.array([[1.2, 2.25, 1.6]])
    x1 = np.array([[1.7, 2.25, 1.6]])
    ora.deposit(x0.T, x1.T, np.array([1.0]), 1.0)
    J = ora.J
    fy, fz = 0.25, 0.6
    assert abs(J[0][1, 2, 1] - 0.5 * (1 - fy) * (1 - fz)) < 1e-15
    assert abs(J[0][1, 3, 1] - 0.5 * fy * (1 - fz)) < 1e-15
    assert abs(J[0][2, 2, 1] - 0.5 * (1 - fy) * fz) < 1e-15
    assert abs(J[0][2, 3, 1] - 0.5 * fy * fz) < 1e-15
    assert abs(J[0].sum() - 0.5) < 1e-15
    assert np.all(J[1] == 0) and np.all(J[2] == 0)


# ---------------------------------------------------------------- FDTD
def _mode(n, d, dt, mvec, e_dir, t_int):
    """Exact discrete Yee plane wave: E at integer time t_int*dt, B at integer
    time (the mean of its two half-step neighbours)."""
    k = np.array([2 * math.pi * mvec[a] / (n[a] * d[a]) for a in range(3)])
    K = np.array([2.0 / d[a] * math.sin(k[a] * d[a] / 2) for a in range(3)])
    e = np.asarray(e_dir, float)
    e = e - K * (K @ e) / (K @ K)
    Om = float(np.linalg.norm(K))
    omega = 2.0 / dt * math.asin(Om * dt / 2)
    b = np.cross(K, e) / Om
    shape = (3, n[2], n[1], n[0])
    E = np.zeros(shape)
    B = np.zeros(shape)
    zz, yy, xx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    t = t_int * dt
    for c in range(3):
        se, sb = bf.STAG_E[c], bf.STAG_B[c]
        ph_e = k[0] * (xx + se[0]) * d[0] + k[1] * (yy + se[1]) * d[1] + k[2] * (zz + se[2]) * d[2]
        ph_b = k[0] * (xx + sb[0]) * d[0] + k[1] * (yy + sb[1]) * d[1] + k[2] * (zz + sb[2]) * d[2]
        E[c] = e[c] * np.cos(ph_e - omega * t)
        B[c] = b[c] * math.cos(omega * dt / 2) * np.cos(ph_b - omega * t)
    return E, B


def _vacuum_steps(ora, nsteps):
    for _ in range(nsteps):
        ora.J[:] = 0
        ora.fdtd_b_half()
        ora.fdtd_e()
        ora.fdtd_b_half()


@pytest.mark.parametrize("mvec,e_dir", [((1, 0, 0), (0, 1, 0)), ((1, 2, 1), (1, -1, 0.5)),
                                         ((0, 1, 3), (1, 0.2, 0.1))])
def test_yee_dispersion_eigenmode(mvec, e_dir):
    n, d = (8, 6, 10), (0.05, 0.06, 0.045)
    dt = 0.9 / math.sqrt(sum(1 / x ** 2 for x in d))
    E, B = _mode(n, d, dt, mvec, e_dir, 0)
    ora = O.Oracle(n, d, dt, E=E, B=B)
    nsteps = 60
    _vacuum_steps(ora, nsteps)
    E1, B1 = _mode(n, d, dt, mvec, e_dir, nsteps)
    assert np.max(np.abs(ora.E - E1)) < 1e-12
    assert np.max(np.abs(ora.B - B1)) < 1e-12


def test_yee_vacuum_energy_invariant():
    n, d = (6, 7, 5), (0.05, 0.05, 0.05)
    dt = 0.5 * d[0] / math.sqrt(3)
    E, B = _rand_fields(n)
    ora = O.Oracle(n, d, dt, E=E, B=B)
    dV = d[0] * d[1] * d[2]

    def W():
        c = bf.curl_E(ora.E, d)
        return 0.5 * dV * (np.sum(ora.E ** 2) + np.sum(ora.B ** 2) - dt ** 2 / 4 * np.sum(c ** 2))

    w0 = W()
    for _ in range(20):
        _vacuum_steps(ora, 10)
        assert abs(W() - w0) < 1e-14 * w0
    # and the plain energy is not conserved exactly (the invariant is not trivial)
    assert abs(ora.field_energy() - 0.5 * dV * (np.sum(E ** 2) + np.sum(B ** 2))) > 1e-8


def test_fdtd_matches_numpy_curls():
    n, d = (5, 4, 6), (0.05, 0.07, 0.04)
    dt = 0.01
    E, B = _rand_fields(n)
    J = RNG.standard_normal(E.shape)
    ora = O.Oracle(n, d, dt, E=E, B=B)
    ora.J[:] = J
    ora.fdtd_b_half()
    ora.fdtd_e()
    B1 = B - 0.5 * dt * bf.curl_E(E, d)
    E1 = E + dt * (bf.curl_B(B1, d) - J)
    assert np.max(np.abs(ora.B - B1)) < 1e-12
    assert np.max(np.abs(ora.E - E1)) < 1e-12


# ---------------------------------------------------------------- whole step
def test_gauss_residual_constant():
    from paper_1608_01009_gb300 import workloads as W
    wl = W.uniform_plasma((6, 6, 8), 4, 0.05, 0.15, seed=7, steps=0)
    ora = O.Oracle.from_workload(wl)
    res0 = ora.div(ora.E) - ora.rho()
    scale = np.max(np.abs(ora.rho()))
    for _ in range(15):
        ora.step(1)
        res = ora.div(ora.E) - ora.rho()
        assert np.max(np.abs(res - res0)) < 1e-11 * scale
    assert np.max(np.abs(ora.E)) > 0  # the plasma did create fields


def test_whole_step_matches_bruteforce():
    n, d = (4, 4, 4), (0.05, 0.05, 0.05)
    dt = 0.5 * d[0] / math.sqrt(3)
    rng = np.random.default_rng(5)
    npart = 8
    L = np.array(n) * np.array(d)
    x = rng.random((npart, 3)) * L
    u = rng.standard_normal((npart, 3)) * 0.3
    w = rng.random(npart) + 0.5
    E, B = _rand_fields(n, 0.5, rng)
    sp = O.OracleSpecies(-1.0, 1.0, x[:, 0], x[:, 1], x[:, 2], u[:, 0], u[:, 1], u[:, 2], w)
    ora = O.Oracle(n, d, dt, E=E, B=B, species=[sp])
    parts = [dict(x=x[i].copy(), u=u[i].copy(), w=w[i]) for i in range(npart)]
    Eb, Bb = E.copy(), B.copy()
    for _ in range(10):
        ora.step(1)
        Eb, Bb, Jb = bf.step(Eb, Bb, n, d, dt, parts, -1.0, 1.0)
        assert np.max(np.abs(ora.J - Jb)) < 1e-12 * np.max(np.abs(Jb))
    assert np.max(np.abs(ora.E - Eb)) < 1e-12 * np.max(np.abs(Eb))
    assert np.max(np.abs(ora.B - Bb)) < 1e-12 * np.max(np.abs(Bb))
    xb = np.array([p["x"] for p in parts])
    ub = np.array([p["u"] for p in parts])
    xo = np.stack([sp.x, sp.y, sp.z], 1)
    dx = (xo - xb + L / 2) % L - L / 2
    assert np.max(np.abs(dx)) < 1e-12 * L.max()
    assert np.max(np.abs(np.stack([sp.ux, sp.uy, sp.uz], 1) - ub)) < 1e-12


# ---------------------------------------------------------------- absorbing
def test_absorbing_layer_removes_pulse():
    from paper_1608_01009_gb300 import workloads as W
    wl = W.laser_slab(n=(4, 4, 64), ppc=1, slab=(0, 0), window=(20, 36), steps=0)
    ora = O.Oracle(wl.n, wl.d, wl.dt, wl.bc, wl.absorb_cells, wl.absorb_sigma, wl.E, wl.B)
    w0 = ora.field_energy()
    # the pulse moves at ~c: 0.2887 cells per step; ~45 cells to cross and enter the layer
    for _ in range(240):
        _vacuum_steps(ora, 1)
    assert ora.field_energy() < 0.05 * w0


def test_absorbing_damping_profile():
    # The layer is a reading (the paper has none): after each field sub-update a
    # component is multiplied by 1 - sigma ((L - dist)/L)^2 inside L cells, dist
    # the distance in cells of the component's own lattice point from the nearer
    # boundary.  With E = 0 the B half step is that factor alone, with B = 0 and
    # J = 0 so is the E update; the x offsets are the Yee staggering (Bx at i,
    # By and Bz at i + 1/2; Ex at i + 1/2, Ey and Ez at i).
    n, d, L, sigma = (24, 4, 4), (0.1, 0.1, 0.1), 8, 0.1
    shape = (3, n[2], n[1], n[0])
    p = np.arange(n[0], dtype=float)

    def factor(off):
        dist = np.minimum(p + off, n[0] - (p + off))
        return np.where(dist < L, 1.0 - sigma * ((L - dist) / L) ** 2, 1.0)

    ora = O.Oracle(n, d, 0.01, bc=(1, 0, 0), absorb_cells=L, absorb_sigma=sigma, E=np.zeros(shape),
                   B=np.ones(shape))
    ora.fdtd_b_half()
    for c, off in enumerate((0.0, 0.5, 0.5)):
        assert np.max(np.abs(ora.B[c] - factor(off)[None, None, :])) < 1e-15, c
    ora = O.Oracle(n, d, 0.01, bc=(1, 0, 0), absorb_cells=L, absorb_sigma=sigma, E=np.ones(shape),
                   B=np.zeros(shape))
    ora.fdtd_e()
    for c, off in enumerate((0.5, 0.0, 0.0)):
        assert np.max(np.abs(ora.E[c] - factor(off)[None, None, :])) < 1e-15, c
    assert abs(factor(0.0)[0] - 0.9) < 1e-15  # the boundary itself: 1 - sigma


def test_absorbing_deactivates_leaving_particles():
    n, d = (4, 4, 16), (0.1, 0.1, 0.1)
    dt = 0.5 * 0.1 / math.sqrt(3)
    sp = O.OracleSpecies(-1.0, 1.0, [0.2, 0.2], [0.2, 0.2], [1.59, 0.01], [0.0, 0.0], [0.0, 0.0],
                         [5.0, -5.0], [1.0, 1.0])
    ora = O.Oracle(n, d, dt, bc=(0, 0, 1), absorb_cells=0, species=[sp])
    ora.step(1)
    assert list(sp.active) == [0, 0]
    z_before = (sp.z[0], sp.z[1])
    ora.step(1)
    assert (sp.z[0], sp.z[1]) == z_before  # inactive particles are frozen
    # nothing is deposited outside the domain and no current flows once they are gone
    ora.step(1)
    assert np.all(ora.J == 0)


# ---------------------------------------------------------------- tangent
def test_tangent_matches_central_differences():
    from paper_1608_01009_gb300 import workloads as W
    wl = W.laser_slab(n=(4, 4, 16), ppc=2, slab=(6, 10), window=(1, 5), wavelength_cells=4, steps=0)
    rng = np.random.default_rng(3)
    vE = rng.standard_normal(wl.E.shape)
    vB = rng.standard_normal(wl.B.shape)
    nsteps = 12

    def run(h):
        w = wl.copy()
        o = O.Oracle(w.n, w.d, w.dt, w.bc, w.absorb_cells, w.absorb_sigma, w.E + h * vE, w.B + h * vB,
                     w.species)
        o.step(nsteps)
        return o.kinetic_energy()

    o = O.Oracle.from_workload(wl.copy())
    Et, Bt = vE.copy(), vB.copy()
    ptan = [[np.zeros(s.n) for _ in range(7)] for s in o.species]
    wk, dwk = o.step_tangent(Et, Bt, ptan, nsteps)
    assert abs(wk - run(0.0)) < 1e-15 * abs(wk) + 1e-300
    # central difference at h = 1e-5: truncation O(h^2) and rounding O(eps / h)
    # both stay far below the 1e-6 bar
    h = 1e-5
    fd = (run(h) - run(-h)) / (2 * h)
    assert abs(fd - dwk) < 1e-6 * abs(dwk)


# ---------------------------------------------------------------- diagnostics
def test_energy_closed_forms():
    # u = (0.75, 0, 0) and (0, 0, 2.4) give gamma = 1.25 and 2.6 exactly.
    sp = O.OracleSpecies(-1.0, 2.0, [0.1, 0.2, 0.3], [0.1] * 3, [0.1] * 3, [0.75, 0.0, 0.3],
                         [0.0, 0.0, 0.4], [0.0, 2.4, 0.0], [3.0, 0.5, 7.0], active=[1, 1, 0])
    ora = O.Oracle((4, 4, 4), (0.1, 0.2, 0.3), 0.01, species=[sp])
    assert abs(ora.kinetic_energy() - 2.0 * (3.0 * 0.25 + 0.5 * 1.6)) < 1e-14
    E = np.zeros((3, 4, 4, 4))
    E[1] = 2.0
    B = np.zeros_like(E)
    B[2] = -1.0
    ora2 = O.Oracle((4, 4, 4), (0.1, 0.2, 0.3), 0.01, E=E, B=B)
    assert abs(ora2.field_energy() - 0.5 * (4.0 + 1.0) * 64 * 0.1 * 0.2 * 0.3) < 1e-14


def test_work_energy_theorem_uniform_e():
    # From rest in a uniform E along x, the kinetic energy gained equals the
    # work q E dx (to O(dt^2) of the leapfrog): m (gamma - 1) = q E x.
    Ex = -0.8
    xs, us, ora = _single_particle_run((Ex, 0, 0), (0, 0, 0), (0, 0, 0), (4.0, 4.0, 4.0), 200, dt=0.005,
                                       n=(64, 4, 4))
    # kinetic energy of u^{N-1/2} against the work done up to the mean of x^{N-1}, x^N
    g = math.sqrt(1 + us[-1] @ us[-1])
    work = -1.0 * Ex * (0.5 * (xs[-1, 0] + xs[-2, 0]) - xs[0, 0])
    assert abs((g - 1.0) - work) < 1e-4 * work
    sp = ora.species[0]
    sp.w[0] = 2.5
    assert abs(ora.kinetic_energy() - 2.5 * (g - 1.0)) < 1e-14


# ---------------------------------------------------------------- threaded timing build
def test_threaded_timing_build_matches_the_serial_oracle():
    # the threaded build (used only to time the oracle on all host cores) runs the
    # same per-particle statements on contiguous particle ranges into private
    # currents; only J's summation order differs, so one step agrees to rounding
    from paper_1608_01009_gb300 import workloads as W
    wl = W.config("c1")
    O.use_threads(False)
    a = O.Oracle.from_workload(wl.copy())
    a.step(1)
    O.use_threads(True)
    try:
        assert O.threads() >= 1
        b = O.Oracle.from_workload(wl.copy())
        b.step(1)
    finally:
        O.use_threads(False)
    for F, G in ((a.E, b.E), (a.B, b.B), (a.J, b.J)):
        assert np.max(np.abs(F - G)) <= 1e-15 * np.max(np.abs(F))
    for k in range(6):
        assert np.array_equal(a.species[0].arr[k], b.species[0].arr[k]), k  # particles: identical statements
