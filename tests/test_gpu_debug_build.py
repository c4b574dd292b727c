"""The index-checking debug build (PICGB_DEBUG=1, libpicgb_debug.so).

Its kernels pass every array index they use through a check that sets a flag
and skips the access when the index falls outside the array, instead of
faulting.  Here: the check fires on its self test; and the small GPU parity
cases (FP64, mixed, second-order form factor, the differentiable path, the
sort with checkpoint/resume) pass against the oracle on that build with the
flags left clear after every test.  The rerun is a child pytest process
because one process loads one build of the library.
"""
import os
import re
import subprocess
import sys

import pytest

from paper_1608_01009_gb300 import build as B
from paper_1608_01009_gb300 import pic as P

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the small cases: whole files whose grids the oracle runs in seconds (the
# cases at the benchmark's sizes, in test_gpu_fullsize.py, are left out)
FILES = ["tests/test_gpu_parity.py", "tests/test_gpu_mixed.py", "tests/test_gpu_tsc.py",
         "tests/test_gpu_adjoint.py", "tests/test_gpu_state.py"]


def _child(code):
    env = dict(os.environ, PICGB_LIBRARY=P.DEBUG_LIB_PATH, PICGB_INDEX_CHECK="1")
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_debug_index_check_fires_and_release_does_not():
    B.build(debug=True)
    r = _child("from paper_1608_01009_gb300 import pic as P; print(P.selftest_index_check(0), P.index_status(0))")
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["-9", "0"], r.stdout
    # the release build compiles the checks out
    assert P.selftest_index_check(0) == 0
    assert P.index_status(0) == 0


def test_parity_cases_pass_on_the_debug_build_with_no_index_outside():
    B.build(debug=True)
    env = dict(os.environ, PICGB_LIBRARY=P.DEBUG_LIB_PATH, PICGB_INDEX_CHECK="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider"] + FILES
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join(r.stdout.splitlines()[-15:])
    assert r.returncode == 0, tail + r.stderr[-2000:]
    m = re.search(r"(\d+) passed", tail)
    assert m and int(m.group(1)) >= 60 and "failed" not in tail, tail
