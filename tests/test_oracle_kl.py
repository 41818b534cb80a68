"""Pins of the oracle's KL minimisation (CPU only).

Pinned by: central differences of the pointwise likelihood derivatives and of
the KL energy along random directions; for a model that is linear in xi (fixed
spectrum, Gaussian likelihood on the field itself) the sample-averaged metric
is the exact Hessian of the energy (checked by differences of the gradient) and
one Newton step with an exact inner solve lands on the Wiener-filter solution
of a dense system built from the cas-sum Hartley matrix written out here;
Newton-CG on Poisson counts lowers the energy at every step and, with a fixed
spectrum, drives the gradient to zero; the metric is symmetric and bounded
below by the identity.
"""
import numpy as np
import pytest

from oracle import amplitude as amp
from oracle.cf import CFModel, matern_fixed_amplitude
from oracle.kl import KLProblem


def _samples(model, S, seed, scale=0.3):
    g = np.random.default_rng(seed)
    half = [scale * g.standard_normal(model.latent_size) for _ in range(S // 2)]
    return half + [-d for d in half]


def _poisson_problem(seed=0):
    m = CFModel((8, 8), (1 / 8, 1 / 8), prior=amp.AmpPrior(n_bins=6))
    g = np.random.default_rng(seed)
    truth = 0.5 * g.standard_normal(m.latent_size)
    data = g.poisson(10.0 * np.exp(m.forward(truth))).astype(np.float64)
    return KLProblem(m, ("poisson", 10.0), data, _samples(m, 4, seed + 1)), g


@pytest.mark.parametrize("lik", [("poisson", 10.0), ("gauss", 0.3, None, "exp"), ("gauss", 0.3, "mask", "identity")])
def test_pointwise_nll_derivative(lik):
    m = CFModel((8,), (1 / 8,), fixed_amp=matern_fixed_amplitude((8,), (1 / 8,)))
    g = np.random.default_rng(3)
    cf = 0.5 * g.standard_normal(8)
    data = g.poisson(10.0, size=8).astype(np.float64) if lik[0] == "poisson" else g.standard_normal(8)
    if lik[0] == "gauss" and lik[2] == "mask":
        lik = ("gauss", 0.3, (g.random(8) < 0.5).astype(np.float64), lik[3])
    p = KLProblem(m, lik, data, [np.zeros(8)])
    h = 1e-6
    for x in range(8):
        e = np.zeros(8)
        e[x] = h
        fd = (p.nll(cf + e) - p.nll(cf - e)) / (2 * h)
        assert abs(fd - p.dnll(cf)[x]) <= 1e-6 * max(1.0, abs(fd))


def test_energy_gradient_central_differences():
    p, g = _poisson_problem()
    xb = 0.2 * g.standard_normal(p.model.latent_size)
    gr = p.gradient(xb)
    for _ in range(3):
        v = g.standard_normal(p.model.latent_size)
        h = 1e-6
        fd = (p.energy(xb + h * v) - p.energy(xb - h * v)) / (2 * h)
        assert abs(fd - gr @ v) <= 1e-6 * max(1.0, abs(fd))


def _linear_gauss(seed=5):
    shape = (8, 4)
    sp = (1 / 8, 1 / 4)
    A = matern_fixed_amplitude(shape, sp, zero_mode=0.7)
    m = CFModel(shape, sp, fixed_amp=A, offset_mean=0.4)
    g = np.random.default_rng(seed)
    mask = (g.random(shape) < 0.6).astype(np.float64)
    data = g.standard_normal(shape)
    p = KLProblem(m, ("gauss", 0.25, mask, "identity"), data, _samples(m, 4, seed + 1))
    return p, A, mask, data, g


@pytest.mark.parametrize("flat_mask", [False, True])
def test_metric_is_exact_hessian_of_linear_gaussian(flat_mask):
    p, A, mask, data, g = _linear_gauss()
    if flat_mask:  # a per-pixel mask given in flat (C) order
        p = KLProblem(p.model, ("gauss", 0.25, mask.ravel(), "identity"), data.ravel(), p.deltas)
    xb = g.standard_normal(p.model.latent_size)
    for _ in range(3):
        v = g.standard_normal(p.model.latent_size)
        h = 1e-3
        fd = (p.gradient(xb + h * v) - p.gradient(xb - h * v)) / (2 * h)
        np.testing.assert_allclose(fd, p.metric_apply(xb, v), rtol=1e-9, atol=1e-9 * np.abs(fd).max())


def test_newton_step_reaches_wiener_filter():
    """Linear model cf = offset + H diag(A) xi, Gaussian noise on cf: the KL's
    minimiser is the posterior mean (I + J^T W J)^-1 J^T W (d - offset) (the
    antithetic residual samples average to zero); J from the cas-sum DHT."""
    p, A, mask, data, g = _linear_gauss()
    n0, n1 = data.shape
    x0, x1 = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    k0, k1 = x0.ravel(), x1.ravel()
    arg = 2 * np.pi * (np.outer(k0, k0) / n0 + np.outer(k1, k1) / n1)
    H = np.cos(arg) + np.sin(arg)
    J = H @ np.diag(A.ravel())
    W = np.diag(mask.ravel() / 0.25 ** 2)
    post = np.linalg.solve(np.eye(J.shape[1]) + J.T @ W @ J, J.T @ W @ (data.ravel() - 0.4))
    xb = g.standard_normal(p.model.latent_size)
    x1_, step, e = p.newton_step(xb, cg_rtol=1e-13, cg_maxiter=500)
    np.testing.assert_allclose(x1_, post, atol=1e-9 * np.abs(post).max())
    assert np.linalg.norm(p.gradient(x1_)) <= 1e-8 * np.linalg.norm(p.gradient(xb))


def test_newton_cg_poisson_decreases_energy():
    """Power-spectrum model: the Fisher metric is not the Hessian of the
    hyper-parameters, so convergence is linear; every accepted step lowers the
    energy and the gradient shrinks."""
    p, g = _poisson_problem(seed=7)
    xb = np.zeros(p.model.latent_size)
    g0 = np.linalg.norm(p.gradient(xb))
    x, it, es = p.minimize(xb, xtol=1e-7, maxiter=35, cg_rtol=1e-8, cg_maxiter=500)
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(es, es[1:]))
    assert np.linalg.norm(p.gradient(x)) <= 1e-2 * g0


def test_newton_cg_poisson_fixed_spectrum_converges():
    """Fixed spectrum, Poisson counts: Newton with the Fisher metric (Gauss-
    Newton for this likelihood) drives the gradient to zero."""
    shape = (16, 8)
    sp = (1 / 16, 1 / 8)
    m = CFModel(shape, sp, fixed_amp=matern_fixed_amplitude(shape, sp, zero_mode=0.5))
    g = np.random.default_rng(11)
    data = g.poisson(10.0 * np.exp(m.forward(0.7 * g.standard_normal(m.latent_size)))).astype(np.float64)
    p = KLProblem(m, ("poisson", 10.0), data, _samples(m, 2, 12))
    xb = np.zeros(m.latent_size)
    g0 = np.linalg.norm(p.gradient(xb))
    x, it, es = p.minimize(xb, xtol=1e-10, maxiter=35, cg_rtol=1e-10, cg_maxiter=1000)
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(es, es[1:]))
    assert np.linalg.norm(p.gradient(x)) <= 1e-8 * g0, (it, np.linalg.norm(p.gradient(x)) / g0)


def test_kl_metric_symmetric_and_above_identity():
    p, g = _poisson_problem(seed=9)
    xb = 0.2 * g.standard_normal(p.model.latent_size)
    u, v = g.standard_normal((2, p.model.latent_size))
    Mu, Mv = p.metric_apply(xb, u), p.metric_apply(xb, v)
    assert abs(Mu @ v - u @ Mv) <= 1e-12 * np.linalg.norm(Mu) * np.linalg.norm(v)
    assert v @ Mv >= v @ v
