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


# ---------------------------------------------------------------- ICR gather pins
#
# With level 0 drawn exactly (Cov s_0 = K0), one refinement
#     s_f = R s_nbhd + L_D xi_f,   R = K_fc K_cc^-1,  L_D L_D^T = K_ff - R K_cf
# reproduces the kernel exactly on every child block and its neighbourhood:
#     Cov(s_f, s_nbhd) = R K_cc = K_fc,   Cov(s_f, s_f) = R K_cc R^T + D = K_ff.
# Both sides are computed below from the oracle's dense linear map, the right-hand
# sides from positions and a Matern-3/2 kernel written out here, and the
# neighbourhood (clamped radial window, periodic angle) and the child order from
# their definitions.  A swapped neighbour order, a different clamp or wrap, or a
# permuted child block breaks an equality by O(1).


def _chart_pos(n0, level, i, j):
    n = n0 * 2 ** level
    u, v = (i + 0.5) / n, (j + 0.5) / n
    r = 0.1 * 10.0 ** u            # r_min (r_max / r_min)^u with r_min = 0.1, r_max = 1
    return np.array([r * np.cos(2 * np.pi * v), r * np.sin(2 * np.pi * v)])


def _matern32(pa, pb, rho):
    d = np.linalg.norm(pa - pb)
    return (1.0 + np.sqrt(3.0) * d / rho) * np.exp(-np.sqrt(3.0) * d / rho)


def _dense_levels(c):
    """Rows of s_0 and s_1 as linear maps of the latent vector (columns = unit xi)."""
    n = c.latent_size
    cols = [c.forward(np.eye(n)[j], return_levels=True) for j in range(n)]
    L0 = np.stack([col[0].ravel() for col in cols], axis=1)
    L1 = np.stack([col[1].ravel() for col in cols], axis=1)
    return L0, L1


@pytest.mark.parametrize("n0,rho", [(4, 0.4), (5, 0.25), (6, 0.15), (6, 0.6)])
def test_icr_one_refinement_reproduces_kernel(n0, rho):
    c = ICRChart(n0=n0, n_levels=1, rho=rho)
    L0, L1 = _dense_levels(c)
    C10 = L1 @ L0.T          # Cov(s_1, s_0)
    C11 = L1 @ L1.T          # Cov(s_1, s_1)
    n1 = 2 * n0
    worst = 0.0
    for i in range(n0):
        w = min(max(i - 1, 0), n0 - 3)          # clamped radial window
        nb = [(w + a, (j_off) % n0) for a in range(3) for j_off in (-1, 0, 1)]
        for j in range(n0):
            nbh = [(r, (j + dj) % n0) for (r, dj) in [(w + a, d) for a in range(3) for d in (-1, 0, 1)]]
            kids = [(2 * i + a, 2 * j + b) for a in range(2) for b in range(2)]
            for (fi, fj) in kids:
                pf = _chart_pos(n0, 1, fi, fj)
                for (ci, cj) in nbh:
                    got = C10[fi * n1 + fj, ci * n0 + cj]
                    exp = _matern32(pf, _chart_pos(n0, 0, ci, cj), rho)
                    worst = max(worst, abs(got - exp))
                for (gi, gj) in kids:
                    got = C11[fi * n1 + fj, gi * n1 + gj]
                    exp = _matern32(pf, _chart_pos(n0, 1, gi, gj), rho)
                    worst = max(worst, abs(got - exp))
        del nb
    assert worst <= 1e-11, worst


def test_icr_one_refinement_detects_outside_neighbours():
    """The identity holds for the 3x3 neighbourhood only: against a coarse pixel
    two radial rows away from an interior child block the covariance is not the
    kernel (so the pin above would see a neighbourhood that is too small or
    shifted)."""
    n0, rho = 6, 0.4
    c = ICRChart(n0=n0, n_levels=1, rho=rho)
    L0, L1 = _dense_levels(c)
    C10 = L1 @ L0.T
    i, j = 2, 3                                  # interior: window rows 1..3
    fi, fj = 2 * i, 2 * j
    ci, cj = 5, j                                # outside the window
    got = C10[fi * 2 * n0 + fj, ci * n0 + cj]
    exp = _matern32(_chart_pos(n0, 1, fi, fj), _chart_pos(n0, 0, ci, cj), rho)
    assert abs(got - exp) > 1e-6


def test_icr_deeper_refinement_conditional_identities():
    """At level 1 -> 2 (level 1 no longer exactly the kernel) the refinement is
    still the conditional step: with C = Cov(s_1) and the neighbourhood /
    children written out here,
        Cov(s_f, s_nbhd) = R C_nn   and   Cov(s_f) - R C_nn R^T = L_D L_D^T."""
    c = ICRChart(n0=4, n_levels=2, rho=0.3)
    n = c.latent_size
    cols = [c.forward(np.eye(n)[k], return_levels=True) for k in range(n)]
    L1 = np.stack([col[1].ravel() for col in cols], axis=1)
    L2 = np.stack([col[2].ravel() for col in cols], axis=1)
    C11, C21, C22 = L1 @ L1.T, L2 @ L1.T, L2 @ L2.T
    R, LD = c.matrices(1)
    nc = 8
    for i in range(nc):
        w = min(max(i - 1, 0), nc - 3)
        for j in (0, 3, nc - 1):
            nb = [(w + a) * nc + (j + d) % nc for a in range(3) for d in (-1, 0, 1)]
            kids = [(2 * i + a) * 2 * nc + 2 * j + b for a in range(2) for b in range(2)]
            Cnn = C11[np.ix_(nb, nb)]
            np.testing.assert_allclose(C21[np.ix_(kids, nb)], R[i] @ Cnn, atol=1e-12)
            resid = C22[np.ix_(kids, kids)] - R[i] @ Cnn @ R[i].T
            np.testing.assert_allclose(resid, LD[i] @ LD[i].T, atol=1e-12)


# ---------------------------------------------------------------- Fisher weight pins
#
# The Fisher metric of a likelihood p(d | cf) in the coordinate cf is
#     w(cf) = E_d[ (d/dcf log p(d | cf))^2 ]  =  E_d[ -d^2/dcf^2 log p(d | cf) ].
# Below both expectations are taken from the densities themselves: the Poisson
# one by summing over its probability mass function, the Gaussian one by
# Gauss-Hermite quadrature of a central-difference second derivative of the
# log-density.


def _poisson_logpmf(d, lam):
    from scipy.special import gammaln
    return d * np.log(lam) - lam - gammaln(d + 1.0)


@pytest.mark.parametrize("cf", [-2.0, -0.3, 0.0, 0.7, 1.5])
def test_poisson_weight_is_fisher_information(cf):
    scale = 10.0
    lam = scale * np.exp(cf)
    d = np.arange(0, int(lam + 40 * np.sqrt(lam) + 60), dtype=np.float64)
    p = np.exp(_poisson_logpmf(d, lam))
    assert abs(p.sum() - 1.0) < 1e-13
    h = 1e-4
    score = (_poisson_logpmf(d, scale * np.exp(cf + h)) - _poisson_logpmf(d, scale * np.exp(cf - h))) / (2 * h)
    fisher = float(np.sum(p * score * score))
    w = poisson_weight(np.array([cf]), scale)[0]
    assert abs(w - fisher) <= 1e-7 * fisher
    assert abs(w - 1.0 / lam) > 0.5 * fisher or lam < 1.5    # not the inverse rate


@pytest.mark.parametrize("response", ["exp", "identity"])
@pytest.mark.parametrize("cf", [-1.0, 0.2, 1.3])
def test_gaussian_weight_is_fisher_information(response, cf):
    sigma = 0.37
    resp = np.exp if response == "exp" else (lambda z: z)

    def logp(d, c):
        return -0.5 * (d - resp(c)) ** 2 / sigma ** 2 - np.log(sigma * np.sqrt(2 * np.pi))

    z, wq = np.polynomial.hermite_e.hermegauss(40)          # nodes for N(0, 1)
    wq = wq / wq.sum()
    d = resp(cf) + sigma * z
    h = 1e-3
    hess = (logp(d, cf + h) - 2 * logp(d, cf) + logp(d, cf - h)) / (h * h)
    fisher = -float(np.sum(wq * hess))
    w = gaussian_weight(np.array([cf]), sigma, response=response)[0]
    assert abs(w - fisher) <= 1e-5 * fisher
    # mask: an unobserved pixel carries no information
    assert gaussian_weight(np.array([cf]), sigma, mask=np.array([0.0]), response=response)[0] == 0.0


@pytest.mark.parametrize("n0,levels", [(8, 3), (4, 4)])
def test_icr_fp64_tolerance_covers_last_bit_inputs(n0, levels):
    """The FP64 ICR parity tolerance (helpers.icr_fp64_tol, from kappa(K_cc))
    bounds how far the oracle itself moves when every chart coordinate changes
    in its last bit, as it may between two independent FP64 assemblies."""
    from helpers import icr_fp64_tol
    tol, _ = icr_fp64_tol(n0, levels)
    eps = np.finfo(np.float64).eps

    class Perturbed(ICRChart):
        def __init__(self, seed, **kw):
            super().__init__(**kw)
            self._g = np.random.default_rng(seed)

        def position(self, level, i, j):
            p = super().position(level, i, j)
            return p * (1 + eps * self._g.choice([-1.0, 0.0, 1.0], size=p.shape))

    base = ICRChart(n0=n0, n_levels=levels)
    g = np.random.default_rng(21)
    xi = g.standard_normal(base.latent_size)
    s0 = base.forward(xi).ravel()
    ct = g.standard_normal(s0.shape)
    v0 = base.vjp(ct)
    for seed in range(3):
        pc = Perturbed(seed, n0=n0, n_levels=levels)
        assert np.abs(pc.forward(xi).ravel() - s0).max() <= tol * np.abs(s0).max()
        assert np.abs(pc.vjp(ct) - v0).max() <= tol * np.abs(v0).max()
