"""Thin ctypes binding over libpicgb.so (C ABI in include/pic.h).

Argument marshalling only: every step of the particle-in-cell path runs in the
library's CUDA kernels.  Device buffers may be torch CUDA tensors (the "_dev"
entry points receive their data pointers) and the context works on the torch
stream it was created with.  If the library has not been built, or no CUDA
device is present, the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpicgb.so")
# the debug build, whose kernels check every array index (PICGB_DEBUG=1)
DEBUG_LIB_PATH = os.path.join(HERE, "libpicgb_debug.so")

PIC_OK = 0
STATUS = {0: "PIC_OK", -1: "PIC_ERR_ARG", -2: "PIC_ERR_CFL", -3: "PIC_ERR_OOM", -4: "PIC_ERR_BIN_OVERFLOW",
          -5: "PIC_ERR_NAN", -6: "PIC_ERR_CUDA", -7: "PIC_ERR_STATE", -8: "PIC_ERR_TIMEOUT",
          -9: "PIC_ERR_INDEX"}
FP64, MIXED = 0, 1
PERIODIC, ABSORBING = 0, 1


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("d", C.c_double * 3), ("dt", C.c_double), ("bc", C.c_int32 * 3),
                ("absorb_cells", C.c_int32), ("absorb_sigma", C.c_double), ("precision", C.c_int32),
                ("supercell", C.c_int32), ("sort_interval", C.c_int32), ("form_factor", C.c_int32),
                ("device", C.c_int32),
                ("stream", C.c_void_p)]


class SpeciesDesc(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("immobile", C.c_int32)]


_VP = C.c_void_p
_P3 = _VP * 3
_lib = None

# name -> argtypes (all return int except pic_last_error)
SIGNATURES = {
    "pic_create": [C.POINTER(GridDesc), C.POINTER(_VP)],
    "pic_destroy": [_VP],
    "pic_last_error": [_VP],
    "pic_add_species": [_VP, C.POINTER(SpeciesDesc), C.c_int64] + [_VP] * 7 + [C.POINTER(C.c_int)],
    "pic_add_species_dev": [_VP, C.POINTER(SpeciesDesc), C.c_int64] + [_VP] * 7 + [C.POINTER(C.c_int)],
    "pic_set_particles": [_VP, C.c_int, C.c_int64] + [_VP] * 7,
    "pic_set_particles_dev": [_VP, C.c_int, C.c_int64] + [_VP] * 7,
    "pic_upload_particles": [_VP, C.c_int, C.c_int64] + [_VP] * 7,
    "pic_set_particles_uploaded": [_VP, C.c_int],
    "pic_count_particles": [_VP, C.c_int, C.POINTER(C.c_int64)],
    "pic_species_info": [_VP, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                         C.POINTER(C.c_int64)],
    "pic_get_state": [_VP, _VP, C.POINTER(C.c_int64)],
    "pic_selftest_wait_timeout": [_VP],
    "pic_set_state": [_VP, _VP, C.c_int64],
    "pic_get_particles": [_VP, C.c_int, C.c_int64, C.POINTER(C.c_int64)] + [_VP] * 8,
    "pic_get_particles_dev": [_VP, C.c_int, C.c_int64, C.POINTER(C.c_int64)] + [_VP] * 8,
    "pic_set_fields": [_VP, _P3, _P3],
    "pic_set_fields_dev": [_VP, _P3, _P3],
    "pic_get_fields": [_VP, _P3, _P3],
    "pic_get_fields_dev": [_VP, _P3, _P3],
    "pic_get_current": [_VP, _P3],
    "pic_get_current_dev": [_VP, _P3],
    "pic_step": [_VP, C.c_int],
    "pic_sync": [_VP],
    "pic_energy": [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "pic_enable_timing": [_VP, C.c_int],
    "pic_stage_times": [_VP, C.POINTER(C.c_double * 4)],
    "pic_launch_count": [_VP, C.POINTER(C.c_int64), C.c_int],
    "pic_field_energy_noalloc": [_P3, _P3, C.POINTER(C.c_int32 * 3), C.POINTER(C.c_double * 3), _VP, _VP],
    "pic_tape_forward": [_VP, C.c_int, C.c_int, C.POINTER(C.c_double)],
    "pic_tape_backward": [_VP, C.c_double, _VP, _VP, _VP, _VP],
    "pic_tape_particle_grad": [_VP, C.c_int, _VP],
    "pic_probe_fp64_fma": [C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "pic_selftest_index_check": [C.c_int],
    "pic_index_status": [C.c_int],
}


def probe_fp64_fma(device: int = 0, iters: int = 2048):
    """Measured FP64 FMA throughput of `device` (pic_probe_fp64_fma):
    returns (TFLOP/s counting an FMA as 2 flops, ms of the timed launch)."""
    lib = load_library()
    tf, ms = C.c_double(), C.c_double()
    rc = lib.pic_probe_fp64_fma(int(device), int(iters), C.byref(tf), C.byref(ms))
    if rc != PIC_OK:
        raise PicError(rc, "pic_probe_fp64_fma failed")
    return tf.value, ms.value


def selftest_index_check(device: int = 0) -> int:
    """Status of the index-check self test (pic_selftest_index_check):
    PIC_ERR_INDEX (-9) in the debug build, PIC_OK (0) in the release build."""
    return int(load_library().pic_selftest_index_check(int(device)))


def index_status(device: int = 0) -> int:
    """pic_index_status: PIC_ERR_INDEX (-9) if a kernel of the debug build saw
    an index outside its array since the last read (flags cleared), else 0."""
    return int(load_library().pic_index_status(int(device)))


def load_library(path: str = None):
    """Load libpicgb.so, or the library PICGB_LIBRARY names (for example the
    debug build, DEBUG_LIB_PATH); raises if it has not been built."""
    global _lib
    if _lib is None:
        path = path or os.environ.get("PICGB_LIBRARY") or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError("libpicgb.so not built: run `python -m paper_1608_01009_gb300.build` "
                               "(the CUDA library is required; there is no CPU fallback)")
        lib = C.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "pic_last_error" else C.c_int
        _lib = lib
    return _lib


def _ptr(a):
    """Data pointer of a numpy array (host) or torch tensor (device)."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def _is_dev(a) -> bool:
    return not isinstance(a, np.ndarray)


class Simulation:
    """One PIC context on one GPU.

    Parameters follow pic_grid_desc (include/pic.h).  Fields are (3, nz, ny, nx)
    arrays, positions physical.  `stream` is a torch.cuda.Stream (default: the
    current stream of `device`).
    """

    def __init__(self, n, d, dt, bc=(PERIODIC,) * 3, precision=FP64, supercell=4, sort_interval=0, device=0,
                 absorb_cells=8, absorb_sigma=0.1, stream=None, form_factor=1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the PIC library runs only on the GPU")
        self.lib = load_library()
        self.torch = torch
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        g = GridDesc()
        for a in range(3):
            g.n[a] = int(n[a])
            g.d[a] = float(d[a])
            g.bc[a] = int(bc[a])
        g.dt = float(dt)
        g.absorb_cells = int(absorb_cells)
        g.absorb_sigma = float(absorb_sigma)
        g.precision = int(precision)
        g.supercell = int(supercell)
        g.sort_interval = int(sort_interval)
        g.form_factor = int(form_factor)
        g.device = int(device)
        g.stream = stream.cuda_stream
        self.desc = g
        self.n, self.d, self.dt = tuple(int(v) for v in n), tuple(float(v) for v in d), float(dt)
        self.precision = precision
        self.ctx = _VP()
        rc = self.lib.pic_create(C.byref(g), C.byref(self.ctx))
        if rc != PIC_OK:
            raise PicError(rc, "pic_create failed (see stderr)")
        self.nspecies = 0
        self._uploads = {}

    # ------------------------------------------------------------------ helpers
    def _check(self, rc):
        if rc != PIC_OK:
            raise PicError(rc, self.lib.pic_last_error(self.ctx).decode())

    def close(self):
        if self.ctx:
            self.lib.pic_destroy(self.ctx)  # waits for both streams
            self.ctx = _VP()
        self._uploads = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def from_workload(cls, wl, precision=FP64, supercell=4, sort_interval=0, device=0, stream=None, form_factor=1):
        sim = cls(wl.n, wl.d, wl.dt, wl.bc, precision, supercell, sort_interval, device, wl.absorb_cells,
                  wl.absorb_sigma, stream, form_factor)
        sim.set_fields(wl.E, wl.B)
        for sp in wl.species:
            sim.add_species(sp.q, sp.m, *sp.arrays())
        return sim

    # ------------------------------------------------------------------ particles
    def add_species(self, q, m, x, y, z, ux, uy, uz, w, immobile=False) -> int:
        """Add a species; immobile=True declares a neutralising background
        (not stored, not pushed, no current)."""
        arrs = [x, y, z, ux, uy, uz, w]
        dev = _is_dev(x)
        if not dev:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        else:
            arrs = [a.contiguous().to(self.torch.float64) for a in arrs]
        n = int(arrs[0].shape[0])
        sid = C.c_int(-1)
        sd = SpeciesDesc(float(q), float(m), 1 if immobile else 0)
        f = self.lib.pic_add_species_dev if dev else self.lib.pic_add_species
        self._check(f(self.ctx, C.byref(sd), n, *[_ptr(a) for a in arrs], C.byref(sid)))
        if dev:
            self.stream.synchronize()
        self.nspecies += 1
        return sid.value

    def species_info(self, species=0) -> dict:
        q, m, imm, nid = C.c_double(), C.c_double(), C.c_int32(), C.c_int64()
        self._check(self.lib.pic_species_info(self.ctx, int(species), C.byref(q), C.byref(m), C.byref(imm),
                                              C.byref(nid)))
        return {"q": q.value, "m": m.value, "immobile": bool(imm.value), "nid": nid.value}

    def get_state(self) -> bytes:
        """The whole simulation state as an opaque byte string (checkpoint)."""
        size = C.c_int64(0)
        self._check(self.lib.pic_get_state(self.ctx, None, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        self._check(self.lib.pic_get_state(self.ctx, buf, C.byref(size)))
        return buf.raw[:size.value]

    def set_state(self, blob: bytes):
        """Restore a state from get_state() of a context with the same grid."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        self._check(self.lib.pic_set_state(self.ctx, buf, len(blob)))
        n = C.c_int64()
        k = 0
        while self.lib.pic_species_info(self.ctx, k, None, None, None, C.byref(n)) == 0:
            k += 1
        self.nspecies = k

    def set_particles(self, species, x, y, z, ux, uy, uz, w):
        arrs = [x, y, z, ux, uy, uz, w]
        dev = _is_dev(x)
        if not dev:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        n = int(arrs[0].shape[0])
        f = self.lib.pic_set_particles_dev if dev else self.lib.pic_set_particles
        self._check(f(self.ctx, int(species), n, *[_ptr(a) for a in arrs]))

    def upload_particles(self, species, x, y, z, ux, uy, uz, w):
        """Start copying a new particle set into the species' upload area
        (asynchronous, on the context's copy stream); set_particles_uploaded
        installs it.  Page-locked host arrays (or device tensors) overlap the
        copy with the running steps; the arrays must stay unchanged until the
        upload has been installed and the context synchronised."""
        arrs = [x, y, z, ux, uy, uz, w]
        if _is_dev(x):
            arrs = [a.contiguous().to(self.torch.float64) for a in arrs]
            self.torch.cuda.current_stream().synchronize()  # the copy stream reads them next
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        n = int(arrs[0].shape[0])
        self._uploads[int(species)] = arrs  # keep the arrays alive while the copy may run
        self._check(self.lib.pic_upload_particles(self.ctx, int(species), n, *[_ptr(a) for a in arrs]))

    def set_particles_uploaded(self, species):
        """Replace the species' particles with the pending upload (asynchronous)."""
        self._check(self.lib.pic_set_particles_uploaded(self.ctx, int(species)))

    def count(self, species=0) -> int:
        n = C.c_int64()
        self._check(self.lib.pic_count_particles(self.ctx, int(species), C.byref(n)))
        return n.value

    def get_particles(self, species=0, device=False):
        """Active particles: dict id, x, y, z, ux, uy, uz, w (numpy, or torch on the GPU)."""
        cap = self.count(species)
        if device:
            t = self.torch
            out = {"id": t.empty(cap, dtype=t.int64, device=self.device)}
            for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
                out[k] = t.empty(cap, dtype=t.float64, device=self.device)
            f = self.lib.pic_get_particles_dev
        else:
            out = {"id": np.empty(cap, np.int64)}
            for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
                out[k] = np.empty(cap, np.float64)
            f = self.lib.pic_get_particles
        n = C.c_int64()
        self._check(f(self.ctx, int(species), cap, C.byref(n), *[_ptr(out[k]) for k in
                                                                   ("id", "x", "y", "z", "ux", "uy", "uz", "w")]))
        return out

    # ------------------------------------------------------------------ fields
    def _field_ptrs(self, F):
        return _P3(*[_ptr(F[c]) for c in range(3)])

    def set_fields(self, E, B):
        dev = _is_dev(E)
        if not dev:
            E = np.ascontiguousarray(E, dtype=np.float64)
            B = np.ascontiguousarray(B, dtype=np.float64)
        f = self.lib.pic_set_fields_dev if dev else self.lib.pic_set_fields
        self._check(f(self.ctx, self._field_ptrs(E), self._field_ptrs(B)))

    def get_fields(self, device=False):
        shape = (3, self.n[2], self.n[1], self.n[0])
        if device:
            E = self.torch.empty(shape, dtype=self.torch.float64, device=self.device)
            B = self.torch.empty_like(E)
            f = self.lib.pic_get_fields_dev
        else:
            E, B = np.empty(shape), np.empty(shape)
            f = self.lib.pic_get_fields
        self._check(f(self.ctx, self._field_ptrs(E), self._field_ptrs(B)))
        return E, B

    def get_current(self, device=False):
        shape = (3, self.n[2], self.n[1], self.n[0])
        if device:
            J = self.torch.empty(shape, dtype=self.torch.float64, device=self.device)
            f = self.lib.pic_get_current_dev
        else:
            J = np.empty(shape)
            f = self.lib.pic_get_current
        self._check(f(self.ctx, self._field_ptrs(J)))
        return J

    # ------------------------------------------------------------------ stepping
    def step(self, nsteps=1):
        self._check(self.lib.pic_step(self.ctx, int(nsteps)))

    def sync(self):
        self._check(self.lib.pic_sync(self.ctx))

    def energy(self):
        wf, wk = C.c_double(), C.c_double()
        self._check(self.lib.pic_energy(self.ctx, C.byref(wf), C.byref(wk)))
        return wf.value, wk.value

    def enable_timing(self, on=True):
        self._check(self.lib.pic_enable_timing(self.ctx, 1 if on else 0))

    def stage_times(self):
        out = (C.c_double * 4)()
        self._check(self.lib.pic_stage_times(self.ctx, C.byref(out)))
        return dict(push_deposit=out[0], field=out[1], sort=out[2], diagnostics=out[3])

    # ------------------------------------------------------------------ differentiable runs
    def tape_forward(self, nsteps, ckpt_every) -> float:
        """Advance nsteps on the differentiable FP64 path, checkpointing every
        ckpt_every steps; returns the final kinetic energy W_K."""
        wk = C.c_double()
        self._check(self.lib.pic_tape_forward(self.ctx, int(nsteps), int(ckpt_every), C.byref(wk)))
        return wk.value

    def tape_backward(self, wk_weight=1.0, gE=None, gB=None):
        """Gradient of wk_weight * W_K + <gE, E_final> + <gB, B_final> with respect
        to the fields at the start of the tape: (dE0, dB0) torch tensors."""
        t = self.torch
        shape = (3, self.n[2], self.n[1], self.n[0])
        dE = t.zeros(shape, dtype=t.float64, device=self.device)
        dB = t.zeros(shape, dtype=t.float64, device=self.device)
        keep = []

        def arr(F):
            if F is None:
                return None
            F = F.contiguous() if not isinstance(F, np.ndarray) else t.as_tensor(F, device=self.device)
            keep.append(F)
            a = _P3(*[F[c].data_ptr() for c in range(3)])
            keep.append(a)
            return C.addressof(a)

        self.stream.synchronize()
        self._check(self.lib.pic_tape_backward(self.ctx, float(wk_weight), arr(gE), arr(gB), arr(dE), arr(dB)))
        return dE, dB

    def tape_particle_grad(self, species=0, n=None):
        """dL/d(x, y, z, ux, uy, uz) of the tape's starting particles, in id order."""
        t = self.torch
        if n is None:
            n = self.species_info(species)["nid"]
        out = [t.zeros(n, dtype=t.float64, device=self.device) for _ in range(6)]
        ptrs = (_VP * 6)(*[o.data_ptr() for o in out])
        self._check(self.lib.pic_tape_particle_grad(self.ctx, int(species), C.addressof(ptrs)))
        return dict(zip(("x", "y", "z", "ux", "uy", "uz"), out))

    def selftest_wait_timeout(self) -> int:
        """Status code of the bounded-wait failure path (PIC_ERR_TIMEOUT = -8 when it works)."""
        return int(self.lib.pic_selftest_wait_timeout(self.ctx))

    def launch_count(self, reset=False) -> int:
        n = C.c_int64()
        self._check(self.lib.pic_launch_count(self.ctx, C.byref(n), 1 if reset else 0))
        return n.value
