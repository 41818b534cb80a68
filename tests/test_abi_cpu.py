"""C-ABI checks that need no GPU: the library loads, exports every function
include/nre.h declares, rejects invalid arguments before touching the device,
and its host-side log-|k| binning equals the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_16683_gb300 import build as b
    b.build()
    from paper_2402_16683_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M):
            if m.group(1) not in ("if", "while", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_boundary():
    names = declared_functions()
    for f in ["cf_create", "cf_forward", "cf_jvp", "cf_vjp", "icr_create", "icr_forward", "icr_jvp",
              "icr_vjp", "lik_create", "metric_create", "metric_apply", "mgvi_rhs", "cg_solve",
              "nre_last_error"]:
        assert f in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2402_16683_gb300 import _lib
    missing = [n for n in declared_functions()
               if n not in _lib.SIGNATURES and n not in ("nre_last_error", "nre_launch_count")]
    assert not missing, missing


@pytest.mark.parametrize("shape,spacing,nb", [
    ((256,), None, 256), ((4096,), None, 256), ((512, 512), None, 256), ((256, 256), None, 256),
    ((1024, 1024), None, 256), ((128, 128, 128), None, 256), ((8, 8), None, 4), ((16, 64), None, 32),
    ((4, 8, 16), None, 16), ((64, 32), (0.5 / 64, 1.0 / 64), 64)])
def test_bin_map_matches_oracle(lib, shape, spacing, nb):
    from oracle.grid import LogBins
    from paper_2402_16683_gb300 import bin_map
    sp = spacing or tuple(1.0 / s for s in shape)
    np.testing.assert_array_equal(bin_map(shape, sp, nb), LogBins(shape, sp, nb).index)


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2402_16683_gb300 import _lib as L
    p = C.c_void_p()
    a = L.CFAmpParams()
    a.kind = L.NRE_AMP_MATERN_FIXED
    a.k0, a.gamma, a.variance = 8.0, 1.5, 1.0
    shp = (C.c_int64 * 1)(6)
    sp = (C.c_double * 1)(1 / 6)
    assert lib.cf_create(C.byref(p), 1, shp, sp, C.byref(a), L.NRE_F32) == L.NRE_EINVAL
    assert b"power of two" in lib.nre_last_error()
    shp2 = (C.c_int64 * 2)(8, 16)
    sp2 = (C.c_double * 2)(1 / 8, 1 / 8)     # unequal total lengths
    assert lib.cf_create(C.byref(p), 2, shp2, sp2, C.byref(a), L.NRE_F32) == L.NRE_EINVAL
    assert b"isotropic" in lib.nre_last_error()
    shp3 = (C.c_int64 * 4)(8, 8, 8, 8)
    sp3 = (C.c_double * 4)(1, 1, 1, 1)
    assert lib.cf_create(C.byref(p), 4, shp3, sp3, C.byref(a), L.NRE_F32) == L.NRE_EINVAL
    assert lib.cf_create(C.byref(p), 1, (C.c_int64 * 1)(8), (C.c_double * 1)(0.125), C.byref(a), 7) == L.NRE_EINVAL
    h = C.c_void_p()
    assert lib.lik_create(C.byref(h), L.NRE_LIK_POISSON, L.NRE_RESP_IDENTITY, None, 0, 10.0) == L.NRE_EINVAL
    assert lib.lik_create(C.byref(h), L.NRE_LIK_GAUSS, L.NRE_RESP_EXP, None, 0, -1.0) == L.NRE_EINVAL
    assert lib.lik_create(C.byref(h), L.NRE_LIK_GAUSS, L.NRE_RESP_EXP, None, 0, 0.1) == L.NRE_OK
    assert lib.lik_destroy(h) == L.NRE_OK
    ch = L.ICRChartParams(5, 0.1, 1.0)
    kp = L.ICRKernelParams(0.1, 1.0)
    assert lib.icr_create(C.byref(p), C.byref(ch), C.byref(kp), 3, L.NRE_F32) == L.NRE_EINVAL
    assert lib.metric_apply(None, None, None, 1, None) == L.NRE_EINVAL
    assert lib.cg_solve(None, None, None, 1, 0.0, 1, None, None, None) == L.NRE_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the header's structs have the C sizes and offsets."""
    import shutil
    import subprocess
    from paper_2402_16683_gb300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"nre_cf_amp_params": L.CFAmpParams, "nre_serve_cfg": L.ServeCfg, "nre_serve_req": L.ServeReq,
               "nre_serve_result": L.ServeResult, "nre_serve_stats": L.ServeStats,
               "icr_chart_params": L.ICRChartParams, "icr_kernel_params": L.ICRKernelParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nre.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_serve_host_side_checks(lib):
    from paper_2402_16683_gb300 import _lib as L
    r = L.ServeReq()
    r.ndim = 2
    r.shape[0], r.shape[1] = 256, 256
    r.amp.kind = L.NRE_AMP_POWER_MODEL
    r.amp.n_bins = 256
    r.n_samples = 8
    r.precond = L.NRE_PRECOND_HARMONIC
    r.response = L.NRE_RESP_EXP
    out = C.c_uint64()
    assert lib.serve_footprint(C.byref(r), L.NRE_F32, C.byref(out)) == L.NRE_OK
    f32 = out.value
    N, lat = 256 * 256, 256 * 256 + 514
    # at least x, b, r, p, q, z of 8 samples and the two sweep intermediates
    assert f32 >= (6 * 8 * lat + 2 * 8 * N) * 4
    assert lib.serve_footprint(C.byref(r), L.NRE_F64, C.byref(out)) == L.NRE_OK
    assert out.value > 1.4 * f32
    r.n_samples = 16
    # eight more samples: at least their x, b, r, p, q, z and sweep intermediates
    assert lib.serve_footprint(C.byref(r), L.NRE_F32, C.byref(out)) == L.NRE_OK
    assert out.value - f32 >= (6 * 8 * lat + 2 * 8 * N) * 4
    r.shape[1] = 100
    assert lib.serve_footprint(C.byref(r), L.NRE_F32, C.byref(out)) == L.NRE_EINVAL
    r.shape[1] = 256
    r.n_samples = 65
    assert lib.serve_footprint(C.byref(r), L.NRE_F32, C.byref(out)) == L.NRE_EINVAL
    r.n_samples = 8
    r.amp.kind = L.NRE_AMP_ARRAY
    assert lib.serve_footprint(C.byref(r), L.NRE_F32, C.byref(out)) == L.NRE_EINVAL
    h = C.c_void_p()
    cfg = L.ServeCfg(0, 0, L.NRE_F32, 8, 1, 0)
    assert lib.serve_create(C.byref(h), C.byref(cfg)) == L.NRE_EINVAL  # max_slots 0
    cfg = L.ServeCfg(0, 4, 5, 8, 1, 0)
    assert lib.serve_create(C.byref(h), C.byref(cfg)) == L.NRE_EINVAL  # dtype
    assert lib.serve_submit(None, None, None) == L.NRE_EINVAL
    assert lib.serve_poll(None, 1, None, 0) == L.NRE_EINVAL
    assert lib.serve_destroy(None) == L.NRE_OK
