"""GPU parity of iterative charted refinement through the C ABI and its
torch.autograd.Function, against the FP64 oracle.

The refinement matrices R, L are assembled independently on each side in FP64;
a last-bit difference of their inputs is amplified by the conditioning of the
9x9 neighbourhood kernel matrices, so the FP64 comparison uses the tolerance
``helpers.icr_fp64_tol`` derives from kappa(K_cc) (1e-12 where that bound is
smaller) and FP32 uses 1e-5 relative to the output's maximum (rel_max).
"""
import numpy as np
import pytest
import torch

import synth
from helpers import DEV, host, icr_fp64_tol, rel_l2, rel_max, rounded
from oracle.icr import ICRChart

pytestmark = pytest.mark.gpu


def _pair(n0, n_levels, dtype, rho=0.1):
    import paper_2402_16683_gb300 as nre
    plan = nre.ICR(n0=n0, n_levels=n_levels, rho=rho, dtype=torch.float64 if dtype == "f64" else torch.float32)
    oc = ICRChart(n0=n0, n_levels=n_levels, rho=rho)
    return plan, oc


def _dev(plan, x):
    return plan.pad(torch.tensor(np.atleast_2d(x), dtype=plan.dtype, device=DEV))


def _timeouts():
    import ctypes as C

    from paper_2402_16683_gb300 import _lib
    n = C.c_uint(0)
    _lib.check(_lib.load().nre_wait_timeouts(C.byref(n), 1))
    return n.value


# (4, 6) and (8, 7): levels of coarse side 64 .. 512 run the adjoint whose fine
# rows arrive by bulk tensor copies (FP64 and FP32); (12, 5): coarse sides 48,
# 96, 192, where the angular wrap falls inside a tile
@pytest.mark.parametrize("n0,levels,dtype", [(8, 3, "f64"), (4, 4, "f64"), (4, 6, "f64"), (8, 7, "f32"),
                                             (12, 5, "f32"), (6, 2, "f32")])
def test_icr_forward_vjp(n0, levels, dtype):
    if dtype == "f64":
        tol, kap = icr_fp64_tol(n0, levels)
        print(f"ICR ({n0}, {levels}) FP64: max kappa(K_cc) per level {['%.2e' % k for k in kap]}, tol {tol:.2e}")
    else:
        tol = 1e-5
    plan, oc = _pair(n0, levels, dtype)
    assert plan.latent_size == oc.latent_size
    g = np.random.default_rng(21)
    B = 2
    xi = rounded(g.standard_normal((B, oc.latent_size)), dtype)
    ct = rounded(g.standard_normal((B, plan.n_out)), dtype)
    s = host(plan.forward(_dev(plan, xi)))
    gr = host(plan.vjp(None, torch.tensor(ct, dtype=plan.dtype, device=DEV)), oc.latent_size)
    jv = host(plan.jvp(None, _dev(plan, xi)))
    for b in range(B):
        ref = oc.forward(xi[b]).ravel()
        assert rel_max(s[b], ref) <= tol
        assert rel_max(jv[b], ref) <= tol
        assert rel_max(gr[b], oc.vjp(ct[b])) <= tol
    assert _timeouts() == 0


def test_icr_autograd_fd_and_oracle_gradient():
    """Config-3 chart (8x8 -> 1024x1024, 7 levels, FP32): backward through the
    autograd.Function equals the oracle gradient; the directional derivative
    matches central differences with step 1e-3; forward-mode AD runs icr_jvp."""
    plan, oc = _pair(8, 7, "f32")
    x = rounded(synth.normal(synth.SEED_POS, oc.latent_size), "f32")
    ct = rounded(synth.normal(synth.SEED_RHS, plan.n_out), "f32")
    xt = _dev(plan, x).requires_grad_(True)
    s = plan(xt)
    (s * torch.tensor(ct[None], dtype=torch.float32, device=DEV)).sum().backward()
    g = host(xt.grad, oc.latent_size)[0]
    assert rel_max(g, oc.vjp(ct)) <= 1e-5
    v = rounded(synth.normal(synth.SEED_TANGENT, oc.latent_size), "f32")
    h = 1e-3
    vp = _dev(plan, v)
    with torch.no_grad():
        fd = (plan(_dev(plan, x) + h * vp) - plan(_dev(plan, x) - h * vp)) / (2 * h)
    jv = host(plan.jvp(None, vp))[0]
    assert rel_max(host(fd)[0], jv) <= 1e-3
    import torch.autograd.forward_ad as fwAD
    with fwAD.dual_level():
        dual = fwAD.make_dual(_dev(plan, x), vp)
        out = fwAD.unpack_dual(plan(dual)).tangent
    assert rel_max(host(out)[0], oc.forward(v).ravel()) <= 1e-5


def test_cf_autograd_fd_and_oracle_gradient():
    from helpers import cf_pair, field_to_dev, to_dev
    plan, om = cf_pair((64, 64), "power", "f32")
    x = rounded(0.5 * synth.normal(synth.SEED_POS, om.latent_size), "f32")
    ct = rounded(synth.normal(synth.SEED_RHS, om.n_field), "f32")
    xt = to_dev(plan, x).requires_grad_(True)
    (plan(xt) * field_to_dev(plan, ct)).sum().backward()
    g = host(xt.grad, om.latent_size)[0]
    ref = om.vjp(x, ct)
    assert rel_max(g[:om.n_field], ref[:om.n_field]) <= 1e-5
    assert rel_max(g[om.n_field:], ref[om.n_field:]) <= 1e-5
    v = rounded(synth.normal(synth.SEED_TANGENT, om.latent_size), "f32")
    h = 1e-3
    with torch.no_grad():
        fd = (plan(to_dev(plan, x + h * v)) - plan(to_dev(plan, x - h * v))) / (2 * h)
    jv = om.jvp(x, v).ravel()
    assert rel_max(host(fd)[0], jv) <= 1e-3


@pytest.mark.parametrize("n0,levels", [(8, 4), (4, 3)])
def test_icr_metric_and_cg(n0, levels):
    """(8, 4): coarse levels fused, the finest refinement (with the weights)
    separate; (4, 3): every level in the fused kernel, weights included."""
    import paper_2402_16683_gb300 as nre
    plan, oc = _pair(n0, levels, "f64")
    lik = nre.Likelihood("gauss", sigma=0.1, response="identity", n_data=plan.n_out)
    xi_p = synth.normal(synth.SEED_POS, oc.latent_size)
    M = nre.Metric(plan, lik, _dev(plan, xi_p)[0], max_batch=2)
    v = np.random.default_rng(3).standard_normal((2, oc.latent_size))
    out = host(M.apply(_dev(plan, v)), oc.latent_size)
    tol, kap = icr_fp64_tol(n0, levels)
    print(f"ICR metric ({n0}, {levels}) FP64: max kappa(K_cc) per level {['%.2e' % k for k in kap]}, tol {tol:.2e}")
    for b in range(2):
        assert rel_max(out[b], oc.metric_apply(v[b], 0.1)) <= tol
    x, its, rel, st = M.cg(_dev(plan, v), rtol=1e-8, maxiter=3000)
    assert st == 0
    xs = host(x, oc.latent_size)
    for b in range(2):
        assert rel_l2(oc.metric_apply(xs[b], 0.1), v[b]) <= 1e-7
