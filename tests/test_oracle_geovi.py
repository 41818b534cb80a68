"""Pins of the oracle's geoVI nonlinear sample update (CPU only).

Pinned by: the standardising transform has unit Fisher information (Poisson by
summation over the probability mass function, Gaussian in closed form through
a central difference of t); J_p^T J_p (J_p by central differences of
xi -> t(cf(xi))) equals the likelihood part of the MGVI metric; for a model
that is linear in xi the linear residual solves the coordinate equation and
the update leaves it unchanged; for Poisson counts the Newton iterations drive
the coordinate residual to zero and move the sample away from the linear one.
"""
import numpy as np
import pytest
from scipy.special import gammaln

from oracle import amplitude as amp
from oracle.cf import CFModel, matern_fixed_amplitude
from oracle.cg import cg
from oracle.geovi import coordinate_residual, nonlinear_update, transform
from oracle.likelihood import gaussian_weight, poisson_weight
from oracle.metric import dense_metric, metric_apply


@pytest.mark.parametrize("cf", [-1.0, 0.4, 1.7])
def test_poisson_transform_has_unit_fisher(cf):
    scale = 10.0
    lam = scale * np.exp(cf)
    d = np.arange(0, int(lam + 40 * np.sqrt(lam) + 60), dtype=np.float64)
    logp = lambda c: d * np.log(scale * np.exp(c)) - scale * np.exp(c) - gammaln(d + 1.0)
    p = np.exp(logp(cf))
    h = 1e-5
    score = (logp(cf + h) - logp(cf - h)) / (2 * h)
    fisher_cf = float(np.sum(p * score * score))
    dt = (transform(("poisson", scale), cf + h)[0] - transform(("poisson", scale), cf - h)[0]) / (2 * h)
    assert abs(fisher_cf / dt ** 2 - 1.0) <= 1e-7
    assert abs(transform(("poisson", scale), cf)[1] - dt) <= 1e-7 * abs(dt)


@pytest.mark.parametrize("resp", ["exp", "identity"])
def test_gaussian_transform_has_unit_fisher(resp):
    sigma, cf = 0.3, 0.8
    h = 1e-5
    t = lambda c: transform(("gauss", sigma, None, resp), np.array([c]))[0][0]
    dt = (t(cf + h) - t(cf - h)) / (2 * h)
    R1 = np.exp(cf) if resp == "exp" else 1.0
    fisher_cf = R1 * R1 / sigma ** 2        # a Gaussian in R(cf) with std sigma
    assert abs(fisher_cf / dt ** 2 - 1.0) <= 1e-8


@pytest.mark.parametrize("lik", [("poisson", 10.0), ("gauss", 0.2, "mask", "exp")])
def test_transform_jacobian_gives_the_metric(lik):
    m = CFModel((8, 4), (1 / 8, 1 / 4), prior=amp.AmpPrior(n_bins=5))
    g = np.random.default_rng(1)
    p = 0.3 * g.standard_normal(m.latent_size)
    if lik[0] == "gauss":
        lik = ("gauss", 0.2, (g.random(m.shape) < 0.5).astype(np.float64), "exp")
        w = gaussian_weight(m.forward(p), 0.2, mask=lik[2], response="exp")
    else:
        w = poisson_weight(m.forward(p), 10.0)
    tfun = lambda xi: transform(lik, m.forward(xi))[0]
    _, dtp = transform(lik, m.forward(p))
    v = g.standard_normal(m.latent_size)
    h = 1e-6
    Jv = (tfun(p + h * v) - tfun(p - h * v)) / (2 * h)
    JtJv = m.vjp(p, dtp * Jv)
    ref = metric_apply(m, p, w, v) - v
    assert np.max(np.abs(JtJv - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_linear_model_keeps_the_linear_sample():
    shape = (8, 8)
    A = matern_fixed_amplitude(shape, (1 / 8, 1 / 8), zero_mode=0.5)
    m = CFModel(shape, (1 / 8, 1 / 8), fixed_amp=A)
    lik = ("gauss", 0.3, None, "identity")
    g = np.random.default_rng(2)
    p = g.standard_normal(m.latent_size)
    w = gaussian_weight(m.forward(p), 0.3, response="identity")
    b = g.standard_normal(m.latent_size)
    d0 = np.linalg.solve(dense_metric(m, p, w), b)
    assert np.max(np.abs(coordinate_residual(m, lik, p, b, d0))) <= 1e-11 * np.max(np.abs(b))
    d, it, steps = nonlinear_update(m, lik, p, w, b, d0, xtol=1e-12, maxiter=5, cg_rtol=1e-13)
    np.testing.assert_allclose(d, d0, atol=1e-10 * np.max(np.abs(d0)))


def test_poisson_update_solves_the_coordinate_equation():
    m = CFModel((16, 8), (1 / 16, 1 / 8), prior=amp.AmpPrior(n_bins=6))
    lik = ("poisson", 10.0)
    g = np.random.default_rng(3)
    p = 0.5 * g.standard_normal(m.latent_size)
    w = poisson_weight(m.forward(p), 10.0)
    b = g.standard_normal(m.latent_size)
    d0, _, _ = cg(lambda v: metric_apply(m, p, w, v), b, rtol=1e-12, maxiter=3000)
    F0 = np.linalg.norm(coordinate_residual(m, lik, p, b, d0))
    d, it, steps = nonlinear_update(m, lik, p, w, b, d0, xtol=1e-10, maxiter=20, cg_rtol=1e-12, cg_maxiter=3000)
    F = np.linalg.norm(coordinate_residual(m, lik, p, b, d))
    assert F <= 1e-6 * F0, (F, F0, steps)
    assert np.linalg.norm(d - d0) >= 1e-3 * np.linalg.norm(d0)
    assert all(b_ <= a_ for a_, b_ in zip(steps, steps[1:]))
