"""Pins of the oracle's amplitude model and correlated field (CPU only).

Pinned by: central finite differences of the hand-written JVP, the adjoint
identity between JVP and VJP, the closed-form covariance of the integrated
Wiener process increments, the normalisation invariant, the pure power law at
zero IWP excitations, the single-mode cas wave and the sample covariance of
the field against the prescribed spectrum.
"""
import numpy as np
import pytest

from oracle import amplitude as amp
from oracle.cf import CFModel, matern_fixed_amplitude
from oracle.grid import LogBins

PRIOR = amp.AmpPrior(n_bins=12)
SHAPE = (8, 12)
SPACING = (1 / 8, 1 / 12)


def _bins():
    return LogBins(SHAPE, SPACING, PRIOR.n_bins)


def test_lognormal_moments():
    mu, s = amp.lognormal_params(1.0, 0.5)
    z = np.random.default_rng(0).standard_normal(400000)
    x = np.exp(mu + s * z)
    assert abs(x.mean() - 1.0) < 4 * 0.5 / np.sqrt(x.size)
    assert abs(x.std() - 0.5) < 0.01


def test_amplitude_jvp_central_differences():
    bins = _bins()
    g = np.random.default_rng(1)
    h = g.standard_normal(PRIOR.n_hyper)
    dh = g.standard_normal(PRIOR.n_hyper)
    eps = 1e-6
    fd = (amp.amplitude(h + eps * dh, PRIOR, bins) - amp.amplitude(h - eps * dh, PRIOR, bins)) / (2 * eps)
    an = amp.jvp(h, dh, PRIOR, bins)
    assert np.max(np.abs(fd - an)) <= 1e-7 * np.max(np.abs(an))


def test_amplitude_vjp_adjoint():
    bins = _bins()
    g = np.random.default_rng(2)
    h = g.standard_normal(PRIOR.n_hyper)
    dh = g.standard_normal(PRIOR.n_hyper)
    gA = g.standard_normal(PRIOR.n_bins)
    lhs = np.dot(amp.jvp(h, dh, PRIOR, bins), gA)
    rhs = np.dot(dh, amp.vjp(h, gA, PRIOR, bins))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_amplitude_normalisation_invariant():
    bins = _bins()
    h = np.random.default_rng(3).standard_normal(PRIOR.n_hyper)
    f = amp.forward(h, PRIOR, bins)
    th_fl = f["theta"][0]
    assert abs(np.sum(bins.counts * f["A"] ** 2) - th_fl ** 2) <= 1e-13 * th_fl ** 2


def test_amplitude_pure_power_law():
    """xi1 = xi2 = 0 leaves x = y = 0: A_b ~ exp(theta_slope (l_b - l_0) / 2)."""
    bins = _bins()
    h = np.zeros(PRIOR.n_hyper)
    h[1] = 0.7
    f = amp.forward(h, PRIOR, bins)
    slope = PRIOR.slope[0] + PRIOR.slope[1] * 0.7
    ratio = f["A"] / f["A"][0]
    np.testing.assert_allclose(ratio, np.exp(slope * (bins.centres - bins.centres[0]) / 2), rtol=1e-13)


def test_iwp_increment_covariance():
    """Increments (dx, dy - D x_{i-1}) have covariance
    theta_flex^2 [[D, D^2/2], [D^2/2, D^3/3 + theta_asp D]] (closed form)."""
    prior = amp.AmpPrior(n_bins=4)
    bins = LogBins((16,), (1 / 16,), 4)
    g = np.random.default_rng(4)
    n = 20000
    i = 2
    D = bins.centres[i] - bins.centres[i - 1]
    samples = np.zeros((n, 2))
    h = np.zeros(prior.n_hyper)
    for t in range(n):
        h[4:] = g.standard_normal(2 * (prior.n_bins - 1))
        f = amp.forward(h, prior, bins)
        x, y = f["x"], f["y"]
        samples[t] = (x[i] - x[i - 1], y[i] - y[i - 1] - D * x[i - 1])
    th_fx, th_as = f["theta"][2], f["theta"][3]
    C = th_fx ** 2 * np.array([[D, D * D / 2], [D * D / 2, D ** 3 / 3 + th_as * D]])
    Ce = np.cov(samples.T)
    # 4-sigma Monte-Carlo bound of each entry: sd(C_ab) ~ sqrt((C_aa C_bb + C_ab^2)/n)
    sd = np.sqrt((np.outer(np.diag(C), np.diag(C)) + C * C) / n)
    assert np.all(np.abs(Ce - C) <= 4 * sd)


def test_single_mode_cas_wave():
    shape = (8, 6)
    k0 = (3, 5)
    A = np.zeros(shape)
    A[k0] = 1.0
    m = CFModel(shape, (1 / 8, 1 / 6), fixed_amp=A)
    s = m.forward(np.ones(m.latent_size))
    x0, x1 = np.meshgrid(np.arange(8), np.arange(6), indexing="ij")
    ang = 2 * np.pi * (k0[0] * x0 / 8 + k0[1] * x1 / 6)
    np.testing.assert_allclose(s, np.cos(ang) + np.sin(ang), atol=1e-14)


def test_fixed_spectrum_normalisation():
    A = matern_fixed_amplitude((256,), (1 / 256,))
    assert A[0] == 0.0
    assert abs(np.sum(A[1:] ** 2) - 1.0) < 1e-14
    np.testing.assert_allclose(A[3] / A[1], ((1 + (3 / 8) ** 2) / (1 + (1 / 8) ** 2)) ** -1.5, rtol=1e-14)
    assert A[5] == A[-5]


def test_field_sample_covariance():
    """Cov(cf_x, cf_y) = sum_k A_k^2 cos(2 pi k (x - y)/N) for the 1-D fixed spectrum."""
    N = 64
    A = matern_fixed_amplitude((N,), (1 / N,))
    m = CFModel((N,), (1 / N,), fixed_amp=A)
    n = 10000
    xi = np.random.default_rng(5).standard_normal((n, N))
    # cf is linear in xi: evaluate its matrix once, then all draws
    Jm = np.stack([m.forward(np.eye(N)[j]) for j in range(N)], axis=1)
    s = xi @ Jm.T
    Ce = (s.T @ s) / n
    k = np.arange(N)
    lag = np.arange(N)
    C = np.array([np.sum(A ** 2 * np.cos(2 * np.pi * k * d / N)) for d in lag])
    for d in [0, 1, 3, 8, 20, 32]:
        sd = np.sqrt((C[0] ** 2 + C[d] ** 2) / n)
        assert abs(Ce[0, d] - C[d]) <= 4 * sd
        assert abs(Ce[5, (5 + d) % N] - C[d]) <= 4 * sd


@pytest.mark.parametrize("kind", ["fixed", "model"])
def test_cf_jvp_fd_and_adjoint(kind):
    shape = (8, 4) if kind == "model" else (16,)
    sp = tuple(1.0 / s for s in shape)
    if kind == "model":
        m = CFModel(shape, sp, prior=amp.AmpPrior(n_bins=6))
    else:
        m = CFModel(shape, sp, fixed_amp=matern_fixed_amplitude(shape, sp))
    g = np.random.default_rng(6)
    xp = g.standard_normal(m.latent_size)
    v = g.standard_normal(m.latent_size)
    ct = g.standard_normal(shape)
    eps = 1e-6
    fd = (m.forward(xp + eps * v) - m.forward(xp - eps * v)) / (2 * eps)
    jv = m.jvp(xp, v)
    assert np.max(np.abs(fd - jv)) <= 1e-7 * np.max(np.abs(jv))
    lhs = np.sum(jv * ct)
    rhs = np.dot(v, m.vjp(xp, ct))
    assert abs(lhs - rhs) <= 1e-13 * np.sqrt(np.sum(jv ** 2) * np.sum(ct ** 2))


def test_cf_offset_mode():
    """The zero mode adds offset_std * xi_0 to every pixel (cas(0) = 1)."""
    prior = amp.AmpPrior(n_bins=6, offset_mean=2.0, offset_std=0.3)
    m = CFModel((8, 8), (1 / 8, 1 / 8), prior=prior)
    xi = np.zeros(m.latent_size)
    xi[0] = 1.5
    np.testing.assert_allclose(m.forward(xi), 2.0 + 0.3 * 1.5, rtol=1e-15)


# ---------------------------------------------------------------- Matern amplitude
#
# Pinned by: central differences of the JVP, the JVP / VJP adjoint identity,
# the normalisation invariant, a flat spectrum at zero slope and far below the
# cutoff, and the power spectrum's log-log slope far above the cutoff (which
# fixes the exponent and its sign).

MPRIOR = amp.MaternPrior(n_bins=12)


def test_matern_jvp_central_differences_and_adjoint():
    bins = _bins()
    g = np.random.default_rng(21)
    h, dh = g.standard_normal((2, 3))
    eps = 1e-6
    fd = (amp.amplitude(h + eps * dh, MPRIOR, bins) - amp.amplitude(h - eps * dh, MPRIOR, bins)) / (2 * eps)
    an = amp.jvp(h, dh, MPRIOR, bins)
    assert np.max(np.abs(fd - an)) <= 1e-7 * np.max(np.abs(an))
    gA = g.standard_normal(MPRIOR.n_bins)
    lhs = np.dot(an, gA)
    rhs = np.dot(dh, amp.vjp(h, gA, MPRIOR, bins))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_matern_normalisation_invariant():
    bins = _bins()
    h = np.random.default_rng(22).standard_normal(3)
    f = amp.forward(h, MPRIOR, bins)
    th_sc = f["theta"][0]
    assert abs(np.sum(bins.counts * f["A"] ** 2) - th_sc ** 2) <= 1e-13 * th_sc ** 2


def test_matern_flat_limits():
    """Zero slope, or a cutoff far above every |k|, gives a flat spectrum
    A_b = theta_scale / sqrt(sum n_b)."""
    bins = _bins()
    mean, std = MPRIOR.loglogslope
    for h in (np.array([0.3, -0.2, -mean / std]), np.array([0.3, 90.0, 0.5])):
        f = amp.forward(h, MPRIOR, bins)
        flat = f["theta"][0] / np.sqrt(bins.counts.sum())
        np.testing.assert_allclose(f["A"], flat, rtol=1e-9)


def test_matern_loglog_slope_above_cutoff():
    """Far above the cutoff the power A^2 falls as |k|^slope."""
    bins = _bins()
    h = np.array([0.0, -60.0, 0.8])       # cutoff ~ 8 exp(-60 s_ln): far below every |k|
    f = amp.forward(h, MPRIOR, bins)
    slope = MPRIOR.loglogslope[0] + MPRIOR.loglogslope[1] * 0.8
    lp = np.log(f["A"] ** 2)
    d = np.diff(lp) / np.diff(bins.centres)
    np.testing.assert_allclose(d, slope, rtol=1e-9)


def test_cf_matern_model_jvp_fd_and_adjoint():
    shape = (8, 4)
    sp = tuple(1.0 / s for s in shape)
    m = CFModel(shape, sp, prior=amp.MaternPrior(n_bins=6))
    assert m.latent_size == 32 + 3
    g = np.random.default_rng(23)
    xp, v = g.standard_normal((2, m.latent_size))
    ct = g.standard_normal(shape)
    eps = 1e-6
    fd = (m.forward(xp + eps * v) - m.forward(xp - eps * v)) / (2 * eps)
    jv = m.jvp(xp, v)
    assert np.max(np.abs(fd - jv)) <= 1e-7 * np.max(np.abs(jv))
    lhs = np.sum(jv * ct)
    rhs = np.dot(v, m.vjp(xp, ct))
    assert abs(lhs - rhs) <= 1e-13 * np.sqrt(np.sum(jv ** 2) * np.sum(ct ** 2))
