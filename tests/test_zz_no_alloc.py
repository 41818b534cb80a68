"""cf_forward_noalloc: the correlated-field forward transform that allocates
no device memory (for callers that cannot call cudaMalloc, e.g. because it may
synchronise the device or because their runtime owns the memory budget).

It must give the same result as cf_forward (the FP32 / FP64 tolerances of the
other GPU tests) on two calls in a row, since every call reuses the same fixed
scratch array, leave the library's and torch's device-memory counts unchanged
on a plan whose workspaces were never grown, and reject a batch that needs
more than that array holds.
This file is collected last, so a run that stops at the first failure has run
every other test before it."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2402_16683_gb300 import build as b
    b.build()
    from paper_2402_16683_gb300 import _lib as L
    return L, L.load()


def _device_bytes(lib):
    v = C.c_int64(-1)
    assert lib.nre_device_bytes(C.byref(v)) == 0
    return v.value


@pytest.mark.parametrize("shape,dtype,tol", [((64, 128), torch.float32, 1e-5),
                                             ((16, 32, 64), torch.float32, 1e-5),
                                             ((256,), torch.float64, 1e-12)])
def test_noalloc_matches_cf_forward(shape, dtype, tol):
    import paper_2402_16683_gb300 as nre
    L, lib = _lib()
    plan = nre.CorrelatedField(shape, amplitude="power", prior=dict(n_bins=64), dtype=dtype)
    g = torch.Generator(device="cuda:0").manual_seed(7)
    B = 3
    xi = plan.pad(torch.randn(B, plan.latent_size, dtype=dtype, device="cuda:0", generator=g))
    ref = plan.forward(xi)
    # a second plan that has never run cf_forward: its workspaces are empty, so
    # any allocation inside the call would show in the library's device bytes
    fresh = nre.CorrelatedField(shape, amplitude="power", prior=dict(n_bins=64), dtype=dtype)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    for out in outs:
        lib_before = _device_bytes(lib)
        torch_before = torch.cuda.memory_allocated()
        rc = lib.cf_forward_noalloc(fresh.handle, C.c_void_p(xi.data_ptr()), C.c_void_p(out.data_ptr()), B, st)
        assert rc == L.NRE_OK, lib.nre_last_error()
        torch.cuda.synchronize()
        assert _device_bytes(lib) == lib_before, "cf_forward_noalloc allocated device memory"
        assert torch.cuda.memory_allocated() == torch_before
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err <= tol, err


def test_noalloc_rejects_oversized_batch():
    import paper_2402_16683_gb300 as nre
    L, lib = _lib()
    plan = nre.CorrelatedField((512, 512), amplitude="power", dtype=torch.float32)
    B = 32   # 32 MiB of intermediates > 16 MiB
    xi = torch.zeros(B, plan.stride, device="cuda:0")
    out = torch.zeros(B, plan.n_field, device="cuda:0")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.cf_forward_noalloc(plan.handle, C.c_void_p(xi.data_ptr()), C.c_void_p(out.data_ptr()), B, st)
    assert rc == L.NRE_EINVAL
    assert b"16777216" in lib.nre_last_error()
