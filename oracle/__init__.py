"""ctypes wrapper of the plain FP64 CPU oracle (oracle/pic_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it.  The product package never imports it, and it never
imports the product package's binding.

Fields are numpy arrays of shape (3, nz, ny, nx) (x fastest); positions are
physical.  Every function follows the passage cited in pic_oracle.cpp.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_oracle

_libs = {}
_threads = False


def use_threads(on: bool = True):
    """Route every following oracle call to the threaded timing build (whole
    steps push the particles on all host cores) or back to the serial build."""
    global _threads
    _threads = bool(on)


def threads() -> int:
    """Host threads a whole step of the current build uses."""
    return int(lib().or_threads())


class OrGrid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("d", C.c_double * 3), ("dt", C.c_double), ("bc", C.c_int * 3),
                ("absorb_cells", C.c_int), ("absorb_sigma", C.c_double), ("form_factor", C.c_int)]


class OrSpecies(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_int64)] + \
               [(k, C.POINTER(C.c_double)) for k in ("x", "y", "z", "ux", "uy", "uz", "w")] + \
               [("active", C.POINTER(C.c_int8))]


_P = C.POINTER(C.c_double)
_PP = C.POINTER(_P)


def lib():
    _lib = _libs.get(_threads)
    if _lib is None:
        _lib = C.CDLL(build_oracle.build(threads=_threads))
        _libs[_threads] = _lib
        G = C.POINTER(OrGrid)
        S = C.POINTER(OrSpecies)
        sig = {
            "or_gather": [G, _PP, _PP, C.c_int64, _P, _P, _P, _P, _P],
            "or_boris": [C.c_int64, _P, _P, _P, C.c_double, C.c_double, C.c_double],
            "or_deposit": [G, _PP, C.c_int64, _P, _P, _P, C.c_double],
            "or_fdtd_b_half": [G, _PP, _PP],
            "or_fdtd_e": [G, _PP, _PP, _PP],
            "or_step": [G, _PP, _PP, _PP, C.c_int, S, C.c_int],
            "or_push_deposit": [G, _PP, _PP, _PP, S],
            "or_field_energy": [G, _PP, _PP],
            "or_kinetic_energy": [S],
            "or_rho": [G, S, _P],
            "or_div": [G, _PP, _P],
            "or_step_tangent": [G, _PP, _PP, _PP, _PP, C.c_int, S, _PP, C.c_int, _P, _P],
        }
        for name, args in sig.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = C.c_double if name in ("or_field_energy", "or_kinetic_energy") else None
        _lib.or_threads.argtypes = []
        _lib.or_threads.restype = C.c_int
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P)


def _pp(arrs):
    ptrs = (_P * len(arrs))(*[_p(a) for a in arrs])
    return ptrs


def make_grid(n, d, dt, bc=(0, 0, 0), absorb_cells=8, absorb_sigma=0.1, form_factor=1) -> OrGrid:
    g = OrGrid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.d[a] = float(d[a])
        g.bc[a] = int(bc[a])
    g.dt = float(dt)
    g.absorb_cells = int(absorb_cells)
    g.absorb_sigma = float(absorb_sigma)
    g.form_factor = int(form_factor)
    return g


class OracleSpecies:
    """Particle arrays of one species, owned as contiguous float64 numpy arrays."""

    def __init__(self, q, m, x, y, z, ux, uy, uz, w, active=None):
        self.q, self.m = float(q), float(m)
        self.arr = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in (x, y, z, ux, uy, uz, w)]
        n = self.arr[0].shape[0]
        self.active = np.ones(n, np.int8) if active is None else np.ascontiguousarray(active, np.int8).copy()

    @classmethod
    def from_species(cls, sp):
        return cls(sp.q, sp.m, sp.x, sp.y, sp.z, sp.ux, sp.uy, sp.uz, sp.w)

    @property
    def n(self):
        return self.arr[0].shape[0]

    x = property(lambda s: s.arr[0])
    y = property(lambda s: s.arr[1])
    z = property(lambda s: s.arr[2])
    ux = property(lambda s: s.arr[3])
    uy = property(lambda s: s.arr[4])
    uz = property(lambda s: s.arr[5])
    w = property(lambda s: s.arr[6])

    def struct(self) -> OrSpecies:
        s = OrSpecies()
        s.q, s.m, s.n = self.q, self.m, self.n
        for k, a in zip(("x", "y", "z", "ux", "uy", "uz", "w"), self.arr):
            setattr(s, k, _p(a))
        s.active = self.active.ctypes.data_as(C.POINTER(C.c_int8))
        return s

    def subset(self, idx):
        return OracleSpecies(self.q, self.m, *[a[idx] for a in self.arr], active=self.active[idx])


class Oracle:
    """Whole PIC state on the host, advanced by the oracle's plain loops."""

    def __init__(self, n, d, dt, bc=(0, 0, 0), absorb_cells=8, absorb_sigma=0.1, E=None, B=None,
                 species=(), form_factor=1):
        self.n, self.d, self.dt, self.bc = tuple(n), tuple(d), float(dt), tuple(bc)
        self.form_factor = int(form_factor)
        self.grid = make_grid(n, d, dt, bc, absorb_cells, absorb_sigma, form_factor)
        shape = (3, n[2], n[1], n[0])
        self.E = np.zeros(shape) if E is None else np.array(E, dtype=np.float64, copy=True)
        self.B = np.zeros(shape) if B is None else np.array(B, dtype=np.float64, copy=True)
        self.J = np.zeros(shape)
        self.species = [s if isinstance(s, OracleSpecies) else OracleSpecies.from_species(s) for s in species]

    @classmethod
    def from_workload(cls, wl, form_factor=1):
        return cls(wl.n, wl.d, wl.dt, wl.bc, wl.absorb_cells, wl.absorb_sigma, wl.E, wl.B, wl.species,
                   form_factor=form_factor)

    def _f(self, F):
        return _pp([F[0], F[1], F[2]])

    def step(self, nsteps=1):
        structs = (OrSpecies * max(1, len(self.species)))(*[s.struct() for s in self.species])
        lib().or_step(C.byref(self.grid), self._f(self.E), self._f(self.B), self._f(self.J),
                      len(self.species), structs, int(nsteps))

    def gather(self, x, y, z):
        n = x.shape[0]
        Eo = np.zeros((3, n))
        Bo = np.zeros((3, n))
        lib().or_gather(C.byref(self.grid), self._f(self.E), self._f(self.B), n,
                        _p(np.ascontiguousarray(x, np.float64)), _p(np.ascontiguousarray(y, np.float64)),
                        _p(np.ascontiguousarray(z, np.float64)), _p(Eo), _p(Bo))
        return Eo, Bo

    def deposit(self, x0, x1, w, q):
        """J += VB current of the moves x0 -> x1 (each 3 x n)."""
        x0 = np.ascontiguousarray(x0, np.float64)
        x1 = np.ascontiguousarray(x1, np.float64)
        lib().or_deposit(C.byref(self.grid), self._f(self.J), x0.shape[1], _p(x0), _p(x1),
                         _p(np.ascontiguousarray(w, np.float64)), float(q))

    def fdtd_b_half(self):
        lib().or_fdtd_b_half(C.byref(self.grid), self._f(self.E), self._f(self.B))

    def fdtd_e(self):
        lib().or_fdtd_e(C.byref(self.grid), self._f(self.E), self._f(self.B), self._f(self.J))

    def push_deposit(self, sp: OracleSpecies):
        """Gather, push, move and deposit one particle set (J is added to)."""
        s = sp.struct()
        lib().or_push_deposit(C.byref(self.grid), self._f(self.E), self._f(self.B), self._f(self.J),
                              C.byref(s))

    def field_energy(self):
        return lib().or_field_energy(C.byref(self.grid), self._f(self.E), self._f(self.B))

    def kinetic_energy(self):
        tot = 0.0
        for s in self.species:
            st = s.struct()
            tot += lib().or_kinetic_energy(C.byref(st))
        return tot

    def rho(self):
        r = np.zeros((self.n[2], self.n[1], self.n[0]))
        for s in self.species:
            st = s.struct()
            lib().or_rho(C.byref(self.grid), C.byref(st), _p(r))
        return r

    def div(self, F):
        out = np.zeros((self.n[2], self.n[1], self.n[0]))
        lib().or_div(C.byref(self.grid), self._f(F), _p(out))
        return out

    def step_tangent(self, E_t, B_t, ptan, nsteps):
        """Forward-mode run.  E_t, B_t: tangents of the fields (3, nz, ny, nx);
        ptan: per species a list of 7 tangent arrays (x,y,z,ux,uy,uz,w).
        Advances the state and returns (W_K, dW_K) at the end, updating the
        tangent arrays in place."""
        structs = (OrSpecies * max(1, len(self.species)))(*[s.struct() for s in self.species])
        flat = [a for lst in ptan for a in lst]
        for a in flat:
            assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        wk = C.c_double()
        dwk = C.c_double()
        lib().or_step_tangent(C.byref(self.grid), self._f(self.E), self._f(self.B), self._f(E_t),
                              self._f(B_t), len(self.species), structs, _pp(flat) if flat else None,
                              int(nsteps), C.byref(wk), C.byref(dwk))
        return wk.value, dwk.value
