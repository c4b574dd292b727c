"""The C-ABI library: builds for sm_103a, loads, exports every entry point that
include/pic.h declares, and validates descriptors on the host (no GPU needed:
validation happens before any CUDA call)."""
import ctypes as C
import math
import os
import re

import pytest

from paper_1608_01009_gb300 import build as B
from paper_1608_01009_gb300 import pic as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^PIC_API\s+[\w\s\*]+?\b(pic_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # and the binding knows every declared entry point
    assert names <= set(P.SIGNATURES)


def test_exports_are_only_the_abi(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == _declared()


def test_debug_build_exports_the_same_abi():
    """The index-checking build (PICGB_DEBUG=1) compiles for sm_103a and
    exports exactly the entry points of the header, like the release build."""
    import subprocess
    path = B.build(debug=True)
    assert path == P.DEBUG_LIB_PATH and os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == _declared()


def _desc(**kw):
    g = P.GridDesc()
    n = kw.get("n", (16, 16, 16))
    d = kw.get("d", (0.05, 0.05, 0.05))
    for a in range(3):
        g.n[a] = n[a]
        g.d[a] = d[a]
        g.bc[a] = kw.get("bc", (0, 0, 0))[a]
    g.dt = kw.get("dt", 0.5 * 0.05 / math.sqrt(3))
    g.absorb_cells = kw.get("absorb_cells", 8)
    g.absorb_sigma = kw.get("absorb_sigma", 0.1)
    g.precision = kw.get("precision", 0)
    g.supercell = kw.get("supercell", 4)
    g.sort_interval = kw.get("sort_interval", 0)
    g.form_factor = kw.get("form_factor", 1)
    g.device = 0
    g.stream = None
    return g


@pytest.mark.parametrize("kw,code", [
    (dict(n=(15, 16, 16)), -1),                 # not a multiple of the supercell
    (dict(n=(2048, 16, 16)), -1),               # beyond the packed-cell range
    (dict(supercell=3), -1),
    (dict(supercell=2, precision=1), -1),       # mixed needs 4 or 8
    (dict(precision=7), -1),
    (dict(d=(0.05, -1.0, 0.05)), -1),
    (dict(dt=0.0), -1),
    (dict(dt=0.05), -2),                        # Courant number 1.73
    (dict(sort_interval=4), -2),                # 4 * 0.2887 >= 1 cell of slack
    (dict(bc=(0, 0, 5)), -1),
    (dict(bc=(0, 0, 1), absorb_cells=9), -1),   # layer wider than half the axis
    (dict(absorb_sigma=1.5), -1),
    (dict(form_factor=3), -1),
    (dict(form_factor=2, precision=1), -1),     # second order runs in FP64 only
])
def test_create_rejects_bad_descriptors(lib, kw, code):
    ctx = C.c_void_p()
    rc = lib.pic_create(C.byref(_desc(**kw)), C.byref(ctx))
    assert rc == code
    assert not ctx.value


def test_null_arguments(lib):
    assert lib.pic_create(None, None) == -1
    assert lib.pic_destroy(None) == -1
    assert lib.pic_step(None, 1) == -1
    assert lib.pic_sync(None) == -1
    assert lib.pic_last_error(None) == b"null context"
    assert lib.pic_upload_particles(None, 0, 0, None, None, None, None, None, None, None) == -1
    assert lib.pic_set_particles_uploaded(None, 0) == -1
