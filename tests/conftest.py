import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _index_flags_clear(request):
    """With PICGB_INDEX_CHECK=1 (the GPU tests rerun on the index-checking
    debug build), every GPU test must also leave the index flags clear."""
    check = os.environ.get("PICGB_INDEX_CHECK") == "1" and request.node.get_closest_marker("gpu")
    if check:
        from paper_1608_01009_gb300 import pic as P
        assert P.selftest_index_check(0) == -9, "not the index-checking build"
    yield
    if check:
        assert P.index_status(0) == 0, "a kernel index fell outside its array (PIC_ERR_INDEX)"
