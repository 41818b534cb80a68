"""Bounded waits of the kernels that stage tiles and rows with bulk copies: a
wait that nothing completes (a barrier expecting bytes that no copy delivers)
runs out after its iteration limit, the kernel counts it and returns, and the
context stays usable.  (Every other GPU test checks that no wait ran out.)"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_wait_that_never_completes_is_counted():
    from paper_2402_16683_gb300 import _lib
    lib = _lib.load()
    n = C.c_uint(0)
    _lib.check(lib.nre_wait_timeouts(C.byref(n), 1))  # clear earlier counts
    _lib.check(lib.nre_wait_selftest(1000, None))
    _lib.check(lib.nre_wait_timeouts(C.byref(n), 1))
    assert n.value == 1
    _lib.check(lib.nre_wait_timeouts(C.byref(n), 0))
    assert n.value == 0
    # the context still runs work after the timed-out kernel
    x = torch.arange(1024, dtype=torch.float32, device="cuda")
    assert float(x.sum()) == 1024 * 1023 / 2
