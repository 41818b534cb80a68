"""GPU parity of the KL minimisation (kl_* through the C ABI) against the FP64
oracle: energy, gradient and sample-averaged metric at a position, one
Newton-CG step, and a minimisation.

Tolerances: FP64 1e-12 relative (rel_max per latent block; the energy
relative to its magnitude), FP32 1e-5 (the FP32 transforms' error).
"""
import numpy as np
import pytest
import torch

from helpers import DEV, blocks_rel, cf_pair, rounded, to_dev
from oracle.kl import KLProblem

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _problem(shape, kind, dtype, lik, S=4, seed=0):
    import paper_2402_16683_gb300 as nre
    plan, om = cf_pair(shape, kind, dtype, n_bins=32)
    g = np.random.default_rng(seed)
    truth = 0.5 * g.standard_normal(om.latent_size)
    n = om.n_field
    mask = None
    if lik == "poisson":
        data = g.poisson(10.0 * np.exp(om.forward(truth))).astype(np.float64)
        L = nre.Likelihood("poisson", scale=10.0)
        olik = ("poisson", 10.0)
    else:
        mask = (g.random(n) < 0.5).astype(np.float64)
        resp = "identity" if lik == "gauss_id" else "exp"
        s = om.forward(truth) if resp == "identity" else np.exp(om.forward(truth))
        data = (s + 0.1 * g.standard_normal(om.shape)).ravel()
        L = nre.Likelihood("gauss", sigma=0.1, mask=mask, response=resp)
        olik = ("gauss", 0.1, mask, resp)
    half = [rounded(0.3 * g.standard_normal(om.latent_size), dtype) for _ in range(S // 2)]
    deltas = np.array(half + [-d for d in half])
    kl = nre.KL(plan, L, data, to_dev(plan, deltas))
    okl = KLProblem(om, olik, data, list(deltas))
    return plan, om, kl, okl, g


CASES = [((32, 32), "power", "poisson"), ((256,), "matern_model", "gauss_exp"), ((8, 16, 16), "power", "gauss_id"),
         ((64, 64), "matern", "poisson")]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,kind,lik", CASES)
def test_kl_energy_gradient_metric(shape, kind, lik, dtype):
    plan, om, kl, okl, g = _problem(shape, kind, dtype, lik)
    xb = rounded(0.2 * g.standard_normal(om.latent_size), dtype)
    e = kl.set_position(to_dev(plan, xb)[0])
    e_ref = okl.energy(xb)
    assert abs(e - e_ref) <= TOL[dtype] * abs(e_ref), (e, e_ref)
    e2, grad = kl.energy_gradient()
    assert e2 == e
    gr = grad.double().cpu().numpy()[:om.latent_size]
    assert blocks_rel(gr, okl.gradient(xb), om.n_field) <= TOL[dtype]
    v = rounded(g.standard_normal(om.latent_size), dtype)
    M = kl.metric()
    out = M.apply(to_dev(plan, v)).double().cpu().numpy()[0, :om.latent_size]
    assert blocks_rel(out, okl.metric_apply(xb, v), om.n_field) <= TOL[dtype]
    # energy at another point leaves the position
    x2 = rounded(xb + 0.1 * g.standard_normal(om.latent_size), dtype)
    assert abs(kl.energy_at(to_dev(plan, x2)[0]) - okl.energy(x2)) <= TOL[dtype] * abs(okl.energy(x2))
    assert torch.equal(kl.position()[:om.latent_size].cpu(), to_dev(plan, xb)[0, :om.latent_size].cpu())


@pytest.mark.parametrize("shape,kind,lik", [((32, 32), "power", "poisson"), ((64, 64), "matern", "poisson")])
def test_kl_newton_step_fp64(shape, kind, lik):
    """One Newton-CG step with a tight inner solve: the new position equals the
    oracle's (same direction up to the CG tolerance, same line-search step)."""
    plan, om, kl, okl, g = _problem(shape, kind, "f64", lik, seed=3)
    xb = 0.2 * g.standard_normal(om.latent_size)
    kl.set_position(to_dev(plan, xb)[0])
    step, e, its = kl.newton_step(cg_rtol=1e-11, cg_maxiter=2000)
    x_ref, st_ref, e_ref = okl.newton_step(xb, cg_rtol=1e-11, cg_maxiter=2000)
    x = kl.position().cpu().numpy()[:om.latent_size]
    assert blocks_rel(x, x_ref, om.n_field) <= 1e-8
    assert abs(step - np.mean(np.abs(st_ref))) <= 1e-8 * max(step, 1e-300)
    assert abs(e - e_ref) <= 1e-11 * abs(e_ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_kl_minimize_fixed_spectrum(dtype):
    """Newton-CG on Poisson counts with a fixed spectrum: the energy falls at
    every step and the gradient vanishes (FP64) or drops by the FP32 floor."""
    plan, om, kl, okl, g = _problem((64, 64), "matern", dtype, "poisson", S=2, seed=5)
    xb = np.zeros(om.latent_size)
    e0 = kl.set_position(to_dev(plan, xb)[0])
    g0 = np.linalg.norm(okl.gradient(xb))
    es = [e0]
    for _ in range(12):
        step, e, its = kl.newton_step(cg_rtol=1e-9 if dtype == "f64" else 1e-5, cg_maxiter=3000)
        es.append(e)
        if step <= (1e-12 if dtype == "f64" else 1e-7):
            break
    assert all(b <= a for a, b in zip(es, es[1:]))
    x = kl.position().double().cpu().numpy()[:om.latent_size]
    gn = np.linalg.norm(okl.gradient(x))
    print(f"{dtype}: energies {es[0]:.6f} -> {es[-1]:.6f} in {len(es) - 1} steps, |grad| {g0:.3e} -> {gn:.3e}")
    assert gn <= (1e-7 if dtype == "f64" else 1e-3) * g0
