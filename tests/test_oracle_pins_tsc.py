"""Pins of the oracle's second-order (TSC) form factor and Esirkepov current.

The TSC form factor is the quadratic B-spline B2(t) = 3/4 - t^2 for |t| < 1/2,
(3/2 - |t|)^2 / 2 for 1/2 <= |t| < 3/2, 0 beyond; Esirkepov's current is the
unique charge-conserving split of the density change into three directional
parts for a product form factor.  Checked here against what the mathematics
fixes (no GPU needed):

* gather  -- exact for uniform and linear fields; the second moment of B2
             adds 1/4: a field x^2 on a lattice interpolates to x^2 + 1/4;
             equal to a direct sum of B2 over every lattice point;
* current -- discrete charge continuity (rho^{n+1} - rho^n)/dt + div J = 0 for
             TSC rho, for moves along all three axes and across cells;
             total current q w d / dt per component for every move;
             the closed form of a move along x that keeps its nearest node:
             J_x(-1/2) = Q d (1 - a - b)/2 Sy Sz, J_x(+1/2) = Q d (1 + a + b)/2 Sy Sz
             (a, b the old and new offsets from the node);
* step    -- the Gauss-law residual div E - rho_TSC stays constant.
"""
import numpy as np
import pytest

import oracle as O
from tests import bruteforce as bf

RNG = np.random.default_rng(20010101)


def b2(t):
    t = np.abs(t)
    return np.where(t < 0.5, 0.75 - t * t, np.where(t < 1.5, 0.5 * (1.5 - t) ** 2, 0.0))


def _lattice_fields(n, fn):
    """E, B with every component f(position of its own staggered lattice point)."""
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    zz, yy, xx = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for c in range(3):
        for F, st, row in ((E, bf.STAG_E, c), (B, bf.STAG_B, 3 + c)):
            F[c] = fn(row, xx + st[c][0], yy + st[c][1], zz + st[c][2])
    return E, B


def test_tsc_gather_uniform_and_linear_exact():
    n, d = (9, 10, 11), (0.1, 0.07, 0.13)
    coef = RNG.standard_normal((6, 4))
    E, B = _lattice_fields(n, lambda r, x, y, z: coef[r, 0] + coef[r, 1] * x + coef[r, 2] * y + coef[r, 3] * z)
    ora = O.Oracle(n, d, 0.01, bc=(1, 1, 1), absorb_cells=0, E=E, B=B, form_factor=2)
    xi = 2.0 + RNG.random((300, 3)) * (np.array(n) - 5)  # 27 lattice neighbours inside
    pos = xi * np.array(d)
    Eo, Bo = ora.gather(pos[:, 0], pos[:, 1], pos[:, 2])
    for c in range(3):
        for got, row in ((Eo[c], c), (Bo[c], 3 + c)):
            want = coef[row, 0] + coef[row, 1] * xi[:, 0] + coef[row, 2] * xi[:, 1] + coef[row, 3] * xi[:, 2]
            assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_tsc_gather_second_moment(axis):
    n, d = (9, 9, 9), (0.1, 0.1, 0.1)
    E, B = _lattice_fields(n, lambda r, x, y, z: (x, y, z)[axis] ** 2)
    ora = O.Oracle(n, d, 0.01, bc=(1, 1, 1), absorb_cells=0, E=E, B=B, form_factor=2)
    xi = 2.0 + RNG.random((200, 3)) * 4.0
    Eo, Bo = ora.gather(*(xi * 0.1).T)
    want = xi[:, axis] ** 2 + 0.25
    for c in range(3):
        assert np.max(np.abs(Eo[c] - want)) < 1e-12
        assert np.max(np.abs(Bo[c] - want)) < 1e-12


def test_tsc_gather_matches_direct_spline_sum():
    n, d = (5, 6, 4), (0.05, 0.07, 0.04)
    E = RNG.standard_normal((3, n[2], n[1], n[0]))
    B = RNG.standard_normal((3, n[2], n[1], n[0]))
    ora = O.Oracle(n, d, 0.01, E=E, B=B, form_factor=2)
    pos = RNG.random((30, 3)) * np.array(n) * np.array(d)
    Eo, Bo = ora.gather(*pos.T)
    xi = pos / np.array(d)
    for p in range(pos.shape[0]):
        for c in range(3):
            for F, st, got in ((E, bf.STAG_E, Eo), (B, bf.STAG_B, Bo)):
                total = 0.0
                # every lattice point, periodic images within reach of the spline
                for k in range(-2, n[2] + 2):
                    wz = b2(xi[p, 2] - (k + st[c][2]))
                    if wz == 0:
                        continue
                    for j in range(-2, n[1] + 2):
                        wy = b2(xi[p, 1] - (j + st[c][1]))
                        if wy == 0:
                            continue
                        for i in range(-2, n[0] + 2):
                            wx = b2(xi[p, 0] - (i + st[c][0]))
                            if wx:
                                total += wx * wy * wz * F[c][k % n[2], j % n[1], i % n[0]]
                assert abs(got[c][p] - total) < 1e-13


def _rho(n, d, dt, q, x, w):
    sp = O.OracleSpecies(q, 1.0, x[:, 0], x[:, 1], x[:, 2], *np.zeros((3, x.shape[0])), w)
    return O.Oracle(n, d, dt, species=[sp], form_factor=2).rho()


@pytest.mark.parametrize("maxstep", [0.3, 0.97])
def test_esirkepov_charge_continuity(maxstep):
    n, d, dt, q = (7, 6, 8), (0.05, 0.04, 0.06), 0.013, -1.0
    npart = 300
    L = np.array(n) * np.array(d)
    x0 = RNG.random((npart, 3)) * L
    x1 = x0 + (RNG.random((npart, 3)) * 2 - 1) * maxstep * np.array(d)
    w = RNG.random(npart) + 0.5
    ora = O.Oracle(n, d, dt, form_factor=2)
    ora.deposit(x0.T, x1.T, w, q)
    r0 = _rho(n, d, dt, q, x0, w)
    r1 = _rho(n, d, dt, q, np.mod(x1, L), w)
    divJ = ora.div(ora.J)
    resid = (r1 - r0) / dt + divJ
    assert np.max(np.abs(divJ)) > 0
    assert np.max(np.abs(resid)) < 1e-13 * np.max(np.abs(divJ))


def test_esirkepov_total_current_is_q_w_d_over_dt():
    n, d, dt, q = (6, 7, 5), (0.05, 0.06, 0.04), 0.01, 1.7
    for _ in range(20):
        x0 = RNG.random((1, 3)) * np.array(n) * np.array(d)
        step = (RNG.random((1, 3)) * 2 - 1) * 0.9 * np.array(d)
        w = np.array([0.3 + RNG.random()])
        ora = O.Oracle(n, d, dt, form_factor=2)
        ora.deposit(x0.T, (x0 + step).T, w, q)
        for c in range(3):
            p, r = (c + 1) % 3, (c + 2) % 3
            want = q * w[0] * (step[0, c] / d[c]) / (dt * d[p] * d[r])
            assert abs(ora.J[c].sum() - want) < 1e-13 * abs(want) + 1e-15


def test_esirkepov_move_along_x_closed_form():
    n, d, dt = (8, 8, 8), (1.0, 1.0, 1.0), 1.0
    x0 = np.array([[3.1, 4.3, 2.8]])          # nearest x node 3, offset a = 0.1
    x1 = np.array([[3.35, 4.3, 2.8]])         # offset b = 0.35, same node
    ora = O.Oracle(n, d, dt, form_factor=2)
    ora.deposit(x0.T, x1.T, np.array([1.0]), 1.0)
    a, bb, dd = 0.1, 0.35, 0.25
    sy = {3: 0.5 * (0.5 - 0.3) ** 2, 4: 0.75 - 0.3 ** 2, 5: 0.5 * (0.5 + 0.3) ** 2}
    sz = {2: 0.5 * (0.5 + 0.2) ** 2, 3: 0.75 - 0.2 ** 2, 4: 0.5 * (0.5 - 0.2) ** 2}
    Jx = ora.J[0]
    want = np.zeros_like(Jx)
    for j, wy in sy.items():
        for k, wz in sz.items():
            want[k, j, 2] = 0.5 * dd * (1 - a - bb) * wy * wz   # edge (2 + 1/2)
            want[k, j, 3] = 0.5 * dd * (1 + a + bb) * wy * wz   # edge (3 + 1/2)
    assert np.max(np.abs(Jx - want)) < 1e-15
    assert np.all(np.abs(ora.J[1]) < 1e-16) and np.all(np.abs(ora.J[2]) < 1e-16)


def test_tsc_gauss_residual_constant():
    from paper_1608_01009_gb300 import workloads as W
    wl = W.uniform_plasma((6, 6, 8), 4, 0.05, 0.2, seed=9, steps=0)
    ora = O.Oracle.from_workload(wl, form_factor=2)
    res0 = ora.div(ora.E) - ora.rho()
    scale = np.max(np.abs(ora.rho()))
    for _ in range(15):
        ora.step(1)
        res = ora.div(ora.E) - ora.rho()
        assert np.max(np.abs(res - res0)) < 1e-11 * scale
    assert np.max(np.abs(ora.E)) > 0
