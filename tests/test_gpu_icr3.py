"""GPU parity of charted refinement on the 3-D spherical log-radial chart
(icr_create with ndim 3) through the C ABI, against the FP64 oracle.

FP64 tolerance: helpers.icr3_fp64_tol, derived from the conditioning of the
27 x 27 neighbourhood kernel matrices that both sides factor independently;
FP32: 1e-5 relative to the output's maximum (rel_max).
"""
import numpy as np
import pytest
import torch

from helpers import DEV, host, icr3_fp64_tol, rel_l2, rel_max, rounded
from oracle.icr3 import ICRChart3D

pytestmark = pytest.mark.gpu


def _pair(n0, levels, dtype, rho):
    import paper_2402_16683_gb300 as nre
    plan = nre.ICR(n0=n0, n_levels=levels, rho=rho, dtype=torch.float64 if dtype == "f64" else torch.float32,
                   ndim=3)
    return plan, ICRChart3D(n0=n0, n_levels=levels, rho=rho)


def _dev(plan, x):
    return plan.pad(torch.tensor(np.atleast_2d(x), dtype=plan.dtype, device=DEV))


# (4, 5) / (8, 3): the FP32 refinement of coarse side 64 runs the kernel that
# takes four coarse voxels per thread
@pytest.mark.parametrize("n0,levels,dtype,rho", [(4, 2, "f64", 0.3), (3, 3, "f64", 0.4), (4, 3, "f32", 0.3),
                                                 (5, 2, "f32", 0.5), (4, 5, "f32", 0.3), (8, 3, "f32", 0.3)])
def test_icr3_forward_jvp_vjp(n0, levels, dtype, rho):
    if dtype == "f64":
        tol, kap = icr3_fp64_tol(n0, levels, rho)
        print(f"3-D ICR ({n0}, {levels}): max kappa(K_cc) per level {['%.2e' % k for k in kap]}, tol {tol:.2e}")
    else:
        tol = 1e-5
    plan, oc = _pair(n0, levels, dtype, rho)
    assert plan.latent_size == oc.latent_size and plan.n_out == oc.sizes[-1] ** 3
    g = np.random.default_rng(31)
    B = 3
    xi = rounded(g.standard_normal((B, oc.latent_size)), dtype)
    ct = rounded(g.standard_normal((B, plan.n_out)), dtype)
    s = host(plan.forward(_dev(plan, xi)))
    jv = host(plan.jvp(None, _dev(plan, xi)))
    gr = host(plan.vjp(None, torch.tensor(ct, dtype=plan.dtype, device=DEV)), oc.latent_size)
    for b in range(B):
        ref = oc.forward(xi[b]).ravel()
        assert rel_max(s[b], ref) <= tol, (b, rel_max(s[b], ref))
        assert rel_max(jv[b], ref) <= tol
        assert rel_max(gr[b], oc.vjp(ct[b])) <= tol, (b, rel_max(gr[b], oc.vjp(ct[b])))


def test_icr3_metric_and_cg():
    import paper_2402_16683_gb300 as nre
    n0, levels, rho = 4, 2, 0.3
    plan, oc = _pair(n0, levels, "f64", rho)
    tol, _ = icr3_fp64_tol(n0, levels, rho)
    lik = nre.Likelihood("gauss", sigma=0.1, response="identity", n_data=plan.n_out)
    xi_p = np.random.default_rng(32).standard_normal(oc.latent_size)
    M = nre.Metric(plan, lik, _dev(plan, xi_p)[0], max_batch=2)
    v = np.random.default_rng(33).standard_normal((2, oc.latent_size))
    out = host(M.apply(_dev(plan, v)), oc.latent_size)
    for b in range(2):
        assert rel_max(out[b], oc.metric_apply(v[b], 0.1)) <= tol
    x, its, rel, st = M.cg(_dev(plan, v), rtol=1e-9, maxiter=5000)
    assert st == 0
    xs = host(x, oc.latent_size)
    for b in range(2):
        assert rel_l2(oc.metric_apply(xs[b], 0.1), v[b]) <= 1e-8


def test_icr3_autograd_gradient():
    plan, oc = _pair(4, 2, "f32", 0.3)
    x = rounded(np.random.default_rng(34).standard_normal(oc.latent_size), "f32")
    ct = rounded(np.random.default_rng(35).standard_normal(plan.n_out), "f32")
    xt = _dev(plan, x).requires_grad_(True)
    (plan(xt) * torch.tensor(ct[None], dtype=torch.float32, device=DEV)).sum().backward()
    assert rel_max(host(xt.grad, oc.latent_size)[0], oc.vjp(ct)) <= 1e-5
