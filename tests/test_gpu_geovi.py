"""GPU parity of the geoVI nonlinear sample update (geovi_update through the C
ABI) against the FP64 oracle.

FP64: from the same starting residuals and with tight inner solves the updated
residuals equal the oracle's to 1e-8 (the inner CG tolerances of both sides);
for a model linear in xi the linear residual stays put.  FP32: the update
reduces the coordinate residual F (evaluated by the oracle in FP64).
"""
import numpy as np
import pytest
import torch

import synth
from helpers import DEV, blocks_rel, cf_pair, host, rounded, to_dev
from oracle.geovi import coordinate_residual, nonlinear_update
from oracle.likelihood import gaussian_weight, poisson_weight

pytestmark = pytest.mark.gpu


def _setup(shape, kind, dtype, lik, seed=1):
    import paper_2402_16683_gb300 as nre
    plan, om = cf_pair(shape, kind, dtype, n_bins=32)
    xi_p = rounded(0.5 * synth.normal(seed, om.latent_size), dtype)
    if lik == "poisson":
        L = nre.Likelihood("poisson", scale=10.0)
        olik = ("poisson", 10.0)
        w = poisson_weight(om.forward(xi_p), 10.0)
    else:
        L = nre.Likelihood("gauss", sigma=0.2, response="identity")
        olik = ("gauss", 0.2, None, "identity")
        w = gaussian_weight(om.forward(xi_p), 0.2, response="identity")
    M = nre.Metric(plan, L, to_dev(plan, xi_p)[0], max_batch=2)
    return plan, om, M, xi_p, w, olik


@pytest.mark.parametrize("shape,kind", [((32, 32), "power"), ((16, 8, 16), "matern_model"), ((512,), "power")])
def test_geovi_update_fp64_matches_oracle(shape, kind):
    plan, om, M, xi_p, w, olik = _setup(shape, kind, "f64", "poisson")
    b = np.random.default_rng(4).standard_normal((2, om.latent_size))
    bd = to_dev(plan, b)
    d0, _, _, st = M.cg(bd, rtol=1e-12, maxiter=5000)
    assert st == 0
    d0h = host(d0, om.latent_size)
    its, steps = M.geovi_update(bd, d0, xtol=0.0, maxiter=4, cg_rtol=1e-12, cg_maxiter=5000)
    d = host(d0, om.latent_size)
    for i in range(2):
        ref, _, osteps = nonlinear_update(om, olik, xi_p, w, b[i], d0h[i], xtol=0.0, maxiter=4, cg_rtol=1e-12,
                                          cg_maxiter=5000)
        print(f"{shape} {kind} system {i}: gpu steps {steps[i]:.3e}, oracle steps {osteps}")
        assert blocks_rel(d[i], ref, om.n_field) <= 1e-8
        assert its[i] == 4


def test_geovi_linear_model_keeps_linear_sample():
    plan, om, M, xi_p, w, olik = _setup((64, 64), "matern", "f64", "gauss")
    b = np.random.default_rng(5).standard_normal((2, om.latent_size))
    bd = to_dev(plan, b)
    d0, _, _, _ = M.cg(bd, rtol=1e-13, maxiter=3000)
    before = d0.clone()
    its, steps = M.geovi_update(bd, d0, xtol=1e-12, maxiter=5, cg_rtol=1e-13, cg_maxiter=3000)
    assert (d0 - before).abs().max().item() <= 1e-10 * before.abs().max().item()
    assert max(steps) <= 1e-12


def test_geovi_update_fp32_reduces_coordinate_residual():
    plan, om, M, xi_p, w, olik = _setup((128, 128), "power", "f32", "poisson")
    b = rounded(np.random.default_rng(6).standard_normal((2, om.latent_size)), "f32")
    bd = to_dev(plan, b)
    d0, _, _, _ = M.cg(bd, rtol=1e-6, maxiter=3000)
    d0h = host(d0, om.latent_size)
    its, steps = M.geovi_update(bd, d0, xtol=1e-6, maxiter=5, cg_rtol=1e-5, cg_maxiter=3000)
    d = host(d0, om.latent_size)
    for i in range(2):
        F0 = np.linalg.norm(coordinate_residual(om, olik, xi_p, b[i], d0h[i]))
        F = np.linalg.norm(coordinate_residual(om, olik, xi_p, b[i], d[i]))
        print(f"system {i}: |F| {F0:.3e} -> {F:.3e} in {its[i]} iterations (|b| {np.linalg.norm(b[i]):.3e})")
        assert F <= 0.05 * F0
