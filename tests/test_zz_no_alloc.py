"""pic_field_energy_noalloc: the field energy for callers that cannot allocate.

Some callers cannot let a library allocate device memory: a framework that
owns all device memory through its own pool, a process that has reserved the
whole device, a latency-critical loop that cannot take cudaMalloc's implicit
synchronisation.  For them pic_field_energy_noalloc computes W_F with its
scratch in a fixed device array.  This file is collected last, so a run that
stops at the first failure has run every other test first; it also passes on
its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1608_01009_gb300 import pic as P
    return P.load_library()


def _noalloc(lib, E, B, n, d, out, stream):
    from paper_1608_01009_gb300 import pic as P
    Ep = P._P3(*[E[c].data_ptr() for c in range(3)])
    Bp = P._P3(*[B[c].data_ptr() for c in range(3)])
    return lib.pic_field_energy_noalloc(Ep, Bp, C.byref((C.c_int32 * 3)(*n)), C.byref((C.c_double * 3)(*d)),
                                        C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))


def test_noalloc_field_energy_matches_pic_energy_and_numpy_twice(lib):
    from paper_1608_01009_gb300 import pic as P
    n, d = (24, 16, 20), (0.05, 0.06, 0.04)
    sim = P.Simulation(n, d, 0.01)
    stream = sim.stream
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(77)
    for call in range(2):
        # a different field each call: the shared scratch keeps the previous call's partials
        E = rng.standard_normal((3, n[2], n[1], n[0])) * (1 + call)
        B = rng.standard_normal((3, n[2], n[1], n[0])) * (2 - call)
        sim.set_fields(E, B)
        wf_ref, _ = sim.energy()  # the existing entry point (pic_energy)
        Ed, Bd = sim.get_fields(device=True)
        stream.synchronize()
        assert _noalloc(lib, Ed, Bd, n, d, out, stream) == P.PIC_OK
        stream.synchronize()
        wf = float(out.item())
        assert abs(wf - wf_ref) <= 1e-12 * abs(wf_ref), (call, wf, wf_ref)
        # and against a value independent of the library: the definition
        # W_F = 1/2 dx dy dz sum (E^2 + B^2), summed by numpy on the host
        wf_np = 0.5 * d[0] * d[1] * d[2] * (float(np.sum(E * E)) + float(np.sum(B * B)))
        assert abs(wf - wf_np) <= 1e-12 * abs(wf_np), (call, wf, wf_np)
    sim.close()


def test_noalloc_rejects_grids_beyond_its_scratch(lib):
    from paper_1608_01009_gb300 import pic as P
    dummy = torch.zeros((3, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = _noalloc(lib, dummy, dummy, (512, 256, 256), (1.0, 1.0, 1.0), out,
                  torch.cuda.current_stream())
    assert rc == -1  # PIC_ERR_ARG: more cells than the fixed scratch holds; nothing is enqueued
