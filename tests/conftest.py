import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(autouse=True)
def _bounded_waits_complete(request):
    """Every GPU test ends with no bounded wait of the kernels run out (the
    device's count of them, reset before the test, is still zero after it;
    the self-test of that count resets it itself)."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    import ctypes as C

    from paper_2402_16683_gb300 import _lib
    lib = _lib.load()
    n = C.c_uint(0)
    _lib.check(lib.nre_wait_timeouts(C.byref(n), 1))
    yield
    _lib.check(lib.nre_wait_timeouts(C.byref(n), 1))
    assert n.value == 0, f"{n.value} bounded waits ran out during the test"
