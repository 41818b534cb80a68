"""Pins of the oracle's metric, MGVI right-hand side, CG and ICR (CPU only).

Pinned by: symmetry and positive definiteness of M, M = I at w = 0, the closed
form M = I + c N A^2 in harmonic space, dense assembly against finite
differences, CG against a dense Cholesky solve, the covariance identities of
the MGVI right-hand side, and for ICR the dense GP conditional computed
through the joint precision matrix, linearity, the adjoint identity and the
sample covariance of the refined field.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import amplitude as amp
from oracle.cf import CFModel, matern_fixed_amplitude
from oracle.cg import cg
from oracle.dht import dht
from oracle.icr import ICRChart
from oracle.likelihood import gaussian_weight, poisson_weight
from oracle.metric import dense_metric, metric_apply, mgvi_rhs


def _model(kind):
    if kind == "model":
        return CFModel((4, 8), (1 / 4, 1 / 8), prior=amp.AmpPrior(n_bins=5))
    return CFModel((16,), (1 / 16,), fixed_amp=matern_fixed_amplitude((16,), (1 / 16,)))


@pytest.mark.parametrize("kind", ["fixed", "model"])
@pytest.mark.parametrize("lik", ["gauss", "poisson"])
def test_metric_symmetric_spd(kind, lik):
    m = _model(kind)
    g = np.random.default_rng(0)
    xp = g.standard_normal(m.latent_size)
    cfp = m.forward(xp)
    w = gaussian_weight(cfp, 0.1) if lik == "gauss" else poisson_weight(cfp, 10.0)
    u = g.standard_normal(m.latent_size)
    v = g.standard_normal(m.latent_size)
    Mu = metric_apply(m, xp, w, u)
    Mv = metric_apply(m, xp, w, v)
    assert abs(np.dot(Mu, v) - np.dot(u, Mv)) <= 1e-12 * np.linalg.norm(Mu) * np.linalg.norm(v)
    assert np.dot(v, Mv) >= np.dot(v, v) * (1 - 1e-14)


def test_metric_zero_weight_is_identity():
    m = _model("model")
    g = np.random.default_rng(1)
    xp = g.standard_normal(m.latent_size)
    v = g.standard_normal(m.latent_size)
    np.testing.assert_allclose(metric_apply(m, xp, np.zeros(m.shape), v), v, rtol=0, atol=0)


def test_metric_closed_form_diagonal():
    """Identity response, fixed A, constant w = c: J = H diag(A) and
    M = I + c diag(A) H H diag(A) = I + c N diag(A^2)."""
    shape = (8, 8)
    A = matern_fixed_amplitude(shape, (1 / 8, 1 / 8), zero_mode=0.4)
    m = CFModel(shape, (1 / 8, 1 / 8), fixed_amp=A)
    c = 3.7
    w = gaussian_weight(np.zeros(shape), 1 / np.sqrt(c), response="identity")
    v = np.random.default_rng(2).standard_normal(m.latent_size)
    expect = v + c * 64 * (A ** 2).ravel() * v
    np.testing.assert_allclose(metric_apply(m, np.zeros(m.latent_size), w, v), expect, rtol=1e-13)


@pytest.mark.parametrize("kind", ["fixed", "model"])
def test_dense_metric_vs_finite_difference_jacobian(kind):
    m = _model(kind)
    g = np.random.default_rng(3)
    xp = g.standard_normal(m.latent_size)
    w = poisson_weight(m.forward(xp))
    n = m.latent_size
    eps = 1e-6
    J = np.zeros((m.n_field, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = eps
        J[:, j] = ((m.forward(xp + e) - m.forward(xp - e)) / (2 * eps)).ravel()
    M_fd = np.eye(n) + J.T @ (w.ravel()[:, None] * J)
    M = dense_metric(m, xp, w)
    assert np.max(np.abs(M - M_fd)) <= 1e-6 * np.max(np.abs(M))


def test_cg_against_cholesky():
    m = _model("fixed")
    g = np.random.default_rng(4)
    xp = g.standard_normal(m.latent_size)
    w = gaussian_weight(m.forward(xp), 0.5)
    M = dense_metric(m, xp, w)
    b = g.standard_normal(m.latent_size)
    x_ref = sla.cho_solve(sla.cho_factor(M), b)
    x, it, rel = cg(lambda p: metric_apply(m, xp, w, p), b, rtol=1e-13, maxiter=200)
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    assert rel <= 1e-13


def test_cg_fixed_iterations_and_rtol():
    m = _model("fixed")
    g = np.random.default_rng(5)
    xp = g.standard_normal(m.latent_size)
    w = gaussian_weight(m.forward(xp), 0.1)
    b = g.standard_normal(m.latent_size)
    mv = lambda p: metric_apply(m, xp, w, p)
    _, it, _ = cg(mv, b, rtol=0.0, maxiter=7)
    assert it == 7
    x, it, rel = cg(mv, b, rtol=1e-5, maxiter=1000)
    assert rel <= 1e-5 and it < 1000
    assert np.linalg.norm(b - mv(x)) <= 1e-4 * np.linalg.norm(b)


def test_cg_exact_on_diagonal():
    """On diag(1, 2, ..., 5) CG terminates in 5 iterations (distinct eigenvalues)."""
    d = np.arange(1.0, 6.0)
    b = np.ones(5)
    x, it, rel = cg(lambda p: d * p, b, rtol=1e-14, maxiter=50)
    assert it <= 5
    np.testing.assert_allclose(x, 1 / d, rtol=1e-12)


def test_mgvi_rhs_covariance():
    """b = xi' + J^T sqrt(w) eta is linear in (xi', eta); with G its matrix,
    Cov b = G G^T must equal M, and samples of M^-1 b have covariance M^-1."""
    m = _model("fixed")
    g = np.random.default_rng(6)
    xp = g.standard_normal(m.latent_size)
    w = gaussian_weight(m.forward(xp), 0.3)
    n, nd = m.latent_size, m.n_field
    G = np.zeros((n, n + nd))
    for j in range(n):
        G[:, j] = mgvi_rhs(m, xp, w, np.eye(n)[j], np.zeros(nd))
    for j in range(nd):
        G[:, n + j] = mgvi_rhs(m, xp, w, np.zeros(n), np.eye(nd)[j])
    M = dense_metric(m, xp, w)
    np.testing.assert_allclose(G @ G.T, M, rtol=1e-12, atol=1e-12 * np.abs(M).max())
    z = g.standard_normal((n + nd, 100000))
    bs = G @ z
    Ce = bs @ bs.T / z.shape[1]
    sd = np.sqrt((np.outer(np.diag(M), np.diag(M)) + M * M) / z.shape[1])
    assert np.all(np.abs(Ce - M) <= 5 * sd)
    xs = np.linalg.solve(M, bs)
    Minv = np.linalg.inv(M)
    Cx = xs @ xs.T / z.shape[1]
    sdx = np.sqrt((np.outer(np.diag(Minv), np.diag(Minv)) + Minv * Minv) / z.shape[1])
    assert np.all(np.abs(Cx - Minv) <= 5 * sdx)


# ---------------------------------------------------------------- ICR


def test_icr_level0_covariance():
    c = ICRChart(n0=5, n_levels=1)
    L = c.L0()
    ii, jj = np.meshgrid(np.arange(5), np.arange(5), indexing="ij")
    p = c.position(0, ii.ravel(), jj.ravel())
    # kernel written out independently of ICRChart.kernel
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    K = (1 + np.sqrt(3) * d / 0.1) * np.exp(-np.sqrt(3) * d / 0.1)
    np.testing.assert_allclose(L @ L.T, K, atol=1e-12)
    assert np.allclose(L, np.tril(L))


@pytest.mark.parametrize("i", [0, 1, 3, 5])
def test_icr_refinement_matches_joint_precision(i):
    """R and D from the joint precision Lambda = K^-1 of (children, neighbourhood):
    Cov(f | c) = Lambda_ff^-1 and E[f | c] = -Lambda_ff^-1 Lambda_fc c."""
    c = ICRChart(n0=6, n_levels=1, rho=0.3)
    R, LD = c.matrices(0)
    pc, pf = c.coarse_fine_points(0, i)
    pts = np.concatenate([pf, pc])
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    K = (1 + np.sqrt(3) * d / 0.3) * np.exp(-np.sqrt(3) * d / 0.3)
    Lam = np.linalg.inv(K)
    Dj = np.linalg.inv(Lam[:4, :4])
    Rj = -Dj @ Lam[:4, 4:]
    np.testing.assert_allclose(R[i], Rj, atol=1e-8)
    np.testing.assert_allclose(LD[i] @ LD[i].T, Dj, atol=1e-9)


def test_icr_window_clamp():
    c = ICRChart(n0=8, n_levels=1)
    assert c.window(0, 0) == 0 and c.window(0, 1) == 0 and c.window(0, 4) == 3
    assert c.window(0, 7) == 5 and c.window(0, 6) == 5


def test_icr_linearity_adjoint():
    c = ICRChart(n0=8, n_levels=3)
    g = np.random.default_rng(7)
    a, b = g.standard_normal((2, c.latent_size))
    al, be = 0.3, -1.7
    np.testing.assert_allclose(c.forward(al * a + be * b), al * c.forward(a) + be * c.forward(b),
                               atol=1e-12)
    ct = g.standard_normal(c.forward(a).shape)
    lhs = np.sum(c.forward(a) * ct)
    rhs = np.dot(a, c.vjp(ct))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_icr_central_differences():
    c = ICRChart(n0=8, n_levels=2)
    g = np.random.default_rng(8)
    x, v = g.standard_normal((2, c.latent_size))
    h = 1e-3
    fd = (c.forward(x + h * v) - c.forward(x - h * v)) / (2 * h)
    np.testing.assert_allclose(fd, c.jvp(v), atol=1e-10)


def test_icr_refined_sample_covariance():
    """Sample covariance of one refinement step equals its dense L L^T."""
    c = ICRChart(n0=4, n_levels=1, rho=0.4)
    n = c.latent_size
    Lm = np.stack([c.forward(np.eye(n)[j]).ravel() for j in range(n)], axis=1)
    C = Lm @ Lm.T
    z = np.random.default_rng(9).standard_normal((n, 50000))
    s = Lm @ z
    Ce = s @ s.T / z.shape[1]
    sd = np.sqrt((np.outer(np.diag(C), np.diag(C)) + C * C) / z.shape[1])
    assert np.all(np.abs(Ce - C) <= 5 * sd)
    # information only: fidelity of ICR to the exact Matern covariance
    ii, jj = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    p = c.position(1, ii.ravel(), jj.ravel())
    K = c.kmat(p, p)
    assert np.max(np.abs(C - K)) < 1.0


def test_icr_metric_spd():
    c = ICRChart(n0=8, n_levels=2)
    g = np.random.default_rng(10)
    u, v = g.standard_normal((2, c.latent_size))
    Mu, Mv = c.metric_apply(u), c.metric_apply(v)
    assert abs(np.dot(Mu, v) - np.dot(u, Mv)) <= 1e-11 * np.linalg.norm(Mu) * np.linalg.norm(v)
    assert np.dot(v, Mv) >= np.dot(v, v)
