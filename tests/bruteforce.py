"""Brute-force restatements used to pin the oracle (tiny inputs only).

Each one computes a stage of the PIC step from a different formulation than
the oracle's, so that a dropped term, a wrong sign or a transposed index in
either shows up as a mismatch:

* gather  -- direct sum of the cloud-in-cell hat function over every lattice
             point (and its periodic images), instead of floor + 8 corners;
* Boris   -- the magnetic half of the Boris step is an exact rotation by
             -2 atan(|t|) about t (a Cayley transform); here it is written
             with Rodrigues' rotation formula instead of the two cross products;
* deposit -- the Villasenor-Buneman edge current is the line integral, along
             the straight move, of the hat weights of the two transverse
             coordinates (the charge passing through each cell face);
             here it is integrated by 3-point Gauss-Legendre quadrature on each
             piece between integer crossings (exact for these quadratic
             integrands), instead of the closed form with the dy dz / 12 term;
* FDTD    -- Yee curls written with numpy rolls on periodic grids.
"""
from __future__ import annotations

import math

import numpy as np

STAG_E = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
STAG_B = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


def hat(s):
    return np.maximum(0.0, 1.0 - np.abs(s))


def _axis_weights(xi, off, n, periodic):
    i = np.arange(n, dtype=np.float64)
    images = (-1, 0, 1) if periodic else (0,)
    return sum(hat(xi - off - i - m * n) for m in images)


def gather(E, B, n, d, pos, bc=(0, 0, 0)):
    """E, B: (3, nz, ny, nx).  pos: (npart, 3) physical.  Returns (npart, 3) x2."""
    out_E = np.zeros((pos.shape[0], 3))
    out_B = np.zeros((pos.shape[0], 3))
    for p in range(pos.shape[0]):
        xi = pos[p] / np.asarray(d)
        for c in range(3):
            for F, stag, out in ((E, STAG_E, out_E), (B, STAG_B, out_B)):
                wx = _axis_weights(xi[0], stag[c][0], n[0], bc[0] == 0)
                wy = _axis_weights(xi[1], stag[c][1], n[1], bc[1] == 0)
                wz = _axis_weights(xi[2], stag[c][2], n[2], bc[2] == 0)
                out[p, c] = np.einsum("kji,i,j,k->", F[c], wx, wy, wz)
    return out_E, out_B


def boris_rodrigues(u, E, B, q, m, dt):
    """One Boris step of one particle, rotation written with Rodrigues' formula."""
    h = 0.5 * q * dt / m
    um = u + h * E
    gm = math.sqrt(1.0 + um @ um)
    t = h * B / gm
    tn = math.sqrt(t @ t)
    if tn == 0.0:
        up = um
    else:
        k = t / tn
        theta = -2.0 * math.atan(tn)
        up = um * math.cos(theta) + np.cross(k, um) * math.sin(theta) + k * (k @ um) * (1 - math.cos(theta))
    return up + h * E


_GL_S = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
_GL_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def deposit(J, n, d, dt, x0, x1, w, q, bc=(0, 0, 0)):
    """Add the charge-conserving current of straight moves x0 -> x1 (physical,
    (npart, 3)) into J (3, nz, ny, nx)."""
    d = np.asarray(d, dtype=np.float64)
    for p in range(x0.shape[0]):
        a = x0[p] / d
        b = x1[p] / d
        dd = b - a
        ts = [0.0, 1.0]
        for ax in range(3):
            if dd[ax] == 0.0:
                continue
            lo, hi = min(a[ax], b[ax]), max(a[ax], b[ax])
            for kk in range(int(math.floor(lo)), int(math.floor(hi)) + 2):
                t = (kk - a[ax]) / dd[ax]
                if 0.0 < t < 1.0:
                    ts.append(t)
        ts = sorted(ts)
        for ta, tb in zip(ts[:-1], ts[1:]):
            if tb <= ta:
                continue
            cell = np.floor(a + 0.5 * (ta + tb) * dd).astype(int)
            for s, gw in zip(_GL_S, _GL_W):
                t = ta + (tb - ta) * 0.5 * (1.0 + s)
                pt = a + t * dd
                wt = gw * 0.5 * (tb - ta)
                for c in range(3):
                    p1, p2 = (c + 1) % 3, (c + 2) % 3
                    Q = q * w[p] / (dt * d[p1] * d[p2])
                    for s1 in (0, 1):
                        for s2 in (0, 1):
                            idx = cell.copy()
                            idx[p1] += s1
                            idx[p2] += s2
                            val = Q * dd[c] * hat(pt[p1] - idx[p1]) * hat(pt[p2] - idx[p2]) * wt
                            ok = True
                            for ax in range(3):
                                if idx[ax] < 0 or idx[ax] >= n[ax]:
                                    if bc[ax] == 0:
                                        idx[ax] %= n[ax]
                                    else:
                                        ok = False
                            if ok:
                                J[c][idx[2], idx[1], idx[0]] += val


def _dfwd(F, ax, dlt):
    # (F(i+1) - F(i)) / d along an array axis (numpy axes: 2 = x, 1 = y, 0 = z)
    return (np.roll(F, -1, axis=ax) - F) / dlt


def _dbwd(F, ax, dlt):
    return (F - np.roll(F, 1, axis=ax)) / dlt


def curl_E(E, d):
    """Forward-difference curl of E onto the B lattice (periodic)."""
    dx, dy, dz = d
    cx = _dfwd(E[2], 1, dy) - _dfwd(E[1], 0, dz)
    cy = _dfwd(E[0], 0, dz) - _dfwd(E[2], 2, dx)
    cz = _dfwd(E[1], 2, dx) - _dfwd(E[0], 1, dy)
    return np.stack([cx, cy, cz])


def curl_B(B, d):
    """Backward-difference curl of B onto the E lattice (periodic)."""
    dx, dy, dz = d
    cx = _dbwd(B[2], 1, dy) - _dbwd(B[1], 0, dz)
    cy = _dbwd(B[0], 0, dz) - _dbwd(B[2], 2, dx)
    cz = _dbwd(B[1], 2, dx) - _dbwd(B[0], 1, dy)
    return np.stack([cx, cy, cz])


def step(E, B, n, d, dt, parts, q, m):
    """One whole periodic step of a list of particles (dicts with x (3,), u (3,), w)."""
    J = np.zeros_like(E)
    pos = np.array([p["x"] for p in parts])
    Ep, Bp = gather(E, B, n, d, pos)
    L = np.asarray(n) * np.asarray(d)
    for i, p in enumerate(parts):
        u = boris_rodrigues(p["u"], Ep[i], Bp[i], q, m, dt)
        g = math.sqrt(1.0 + u @ u)
        x1 = p["x"] + dt * u / g
        deposit(J, n, d, dt, p["x"][None, :], x1[None, :], np.array([p["w"]]), q)
        p["u"] = u
        p["x"] = np.mod(x1, L)
    B = B - 0.5 * dt * curl_E(E, d)
    E = E + dt * (curl_B(B, d) - J)
    B = B - 0.5 * dt * curl_E(E, d)
    return E, B, J
