"""Non-parametric amplitude model sqrt(P) (oracle; test infrastructure only).

Sec. "Gaussian Processes" builds sqrt(P) from the ``add_fluctuations`` parameters
``fluctuations``, ``loglogavgslope``, ``flexibility`` and ``asperity`` (each a
(mean, std) pair) and an offset with (mean, std), ``non_parametric_kind="power"``.
The paper defers the equations to its citations, so the model below is the
reading used throughout this project, written step by step in float64:

1. Hyper-parameters from standard-normal excitations (standardization, Sec.
   "Core Components"): fluctuations, flexibility and asperity are log-normal with
   the given mean m and std s of the variable itself,
       mu = ln(m^2 / sqrt(m^2 + s^2)),  s_ln = sqrt(ln(1 + s^2/m^2)),
       theta = exp(mu + s_ln xi);
   the slope is normal, theta_slope = m + s xi.
2. Integrated Wiener process on the log-|k| bin centres l_0..l_{B-1} with steps
   D_i = l_i - l_{i-1}, i = 1..B-1, excitations xi1_i, xi2_i (x_0 = y_0 = 0):
       x_i = x_{i-1} + theta_flex sqrt(D_i) xi1_i
       y_i = y_{i-1} + D_i (x_{i-1} + x_i)/2
                     + theta_flex sqrt(D_i^3/12 + theta_asp D_i) xi2_i
   (D^3/12 is the Brownian-bridge variance of the integral; asperity adds a
   Wiener term to the integrated process).
3. Log-power tau_i = theta_slope (l_i - l_0) + y_i, a_i = exp(tau_i / 2).
4. Normalisation over the non-zero modes of the grid, with n_b modes in bin b:
       S = sum_b n_b a_b^2,   A_b = theta_fluct a_b / sqrt(S),
   so that the pointwise field variance without the zero mode is theta_fluct^2.

Hyper-latent layout h = [xi_fluct, xi_slope, xi_flex, xi_asp,
xi1_1..xi1_{B-1}, xi2_1..xi2_{B-1}], of size 4 + 2 (B - 1).

The parametric alternative, the Matern amplitude of the same section (the
paper names it beside the non-parametric kernel and defers its form to its
citations), is read here as a Matern-type power spectrum on the same log-|k|
bins, evaluated at the bin-centre wavenumbers k_b = exp(l_b):

1. theta_scale and theta_cutoff log-normal, theta_slope normal, from
   standard-normal excitations as in step 1 above;
2. a_b = (1 + (k_b / theta_cutoff)^2)^(theta_slope / 4), so that the power
   a_b^2 falls off with log-log slope theta_slope far above the cutoff and is
   flat below it;
3. A_b = theta_scale a_b / sqrt(sum_b n_b a_b^2) (pointwise field variance
   without the zero mode theta_scale^2).

Hyper-latent layout h = [xi_scale, xi_cutoff, xi_slope].
"""
import numpy as np


class AmpPrior:
    """Prior (mean, std) pairs of the amplitude model and of the offset."""

    def __init__(self, fluct=(1.0, 0.5), slope=(-3.0, 0.5), flex=(1.0, 0.5),
                 asp=(0.1, 0.05), offset_mean=0.0, offset_std=1.0, n_bins=256):
        self.fluct = tuple(map(float, fluct))
        self.slope = tuple(map(float, slope))
        self.flex = tuple(map(float, flex))
        self.asp = tuple(map(float, asp))
        self.offset_mean = float(offset_mean)
        self.offset_std = float(offset_std)
        self.n_bins = int(n_bins)

    @property
    def n_hyper(self):
        return 4 + 2 * (self.n_bins - 1)


class MaternPrior:
    """Prior (mean, std) pairs of the parametric Matern amplitude and of the
    offset: scale and cutoff log-normal, loglogslope normal."""

    def __init__(self, scale=(1.0, 0.5), cutoff=(8.0, 2.0), loglogslope=(-4.0, 0.5),
                 offset_mean=0.0, offset_std=1.0, n_bins=256):
        self.scale = tuple(map(float, scale))
        self.cutoff = tuple(map(float, cutoff))
        self.loglogslope = tuple(map(float, loglogslope))
        self.offset_mean = float(offset_mean)
        self.offset_std = float(offset_std)
        self.n_bins = int(n_bins)

    @property
    def n_hyper(self):
        return 3


def lognormal_params(mean, std):
    """(mu, s_ln) of a log-normal variable with the given mean and std."""
    mu = np.log(mean * mean / np.sqrt(mean * mean + std * std))
    s_ln = np.sqrt(np.log(1.0 + std * std / (mean * mean)))
    return mu, s_ln


def _split(h, nb):
    h = np.asarray(h, dtype=np.float64)
    assert h.shape == (4 + 2 * (nb - 1),)
    return h[0], h[1], h[2], h[3], h[4:4 + nb - 1], h[4 + nb - 1:]


def _thetas(h, prior):
    nb = prior.n_bins
    e_fl, e_sl, e_fx, e_as, xi1, xi2 = _split(h, nb)
    mu_fl, s_fl = lognormal_params(*prior.fluct)
    mu_fx, s_fx = lognormal_params(*prior.flex)
    mu_as, s_as = lognormal_params(*prior.asp)
    th_fl = np.exp(mu_fl + s_fl * e_fl)
    th_sl = prior.slope[0] + prior.slope[1] * e_sl
    th_fx = np.exp(mu_fx + s_fx * e_fx)
    th_as = np.exp(mu_as + s_as * e_as)
    return (th_fl, th_sl, th_fx, th_as), (s_fl, prior.slope[1], s_fx, s_as), xi1, xi2


def forward(h, prior, bins):
    """Amplitude per bin A_b (float64, length n_bins) and the intermediates."""
    if isinstance(prior, MaternPrior):
        return matern_forward(h, prior, bins)
    nb = prior.n_bins
    (th_fl, th_sl, th_fx, th_as), _, xi1, xi2 = _thetas(h, prior)
    l = bins.centres
    x = np.zeros(nb)
    y = np.zeros(nb)
    c = np.zeros(nb)
    for i in range(1, nb):
        d = l[i] - l[i - 1]
        x[i] = x[i - 1] + th_fx * np.sqrt(d) * xi1[i - 1]
        c[i] = np.sqrt(d ** 3 / 12.0 + th_as * d)
        y[i] = y[i - 1] + d * (x[i - 1] + x[i]) / 2.0 + th_fx * c[i] * xi2[i - 1]
    tau = th_sl * (l - l[0]) + y
    a = np.exp(tau / 2.0)
    S = np.sum(bins.counts * a * a)
    A = th_fl * a / np.sqrt(S)
    return dict(A=A, a=a, S=S, x=x, y=y, c=c, tau=tau,
                theta=(th_fl, th_sl, th_fx, th_as))


def amplitude(h, prior, bins):
    return forward(h, prior, bins)["A"]


def jvp(h, dh, prior, bins):
    """Forward-mode derivative dA_b of the amplitude in direction ``dh``."""
    if isinstance(prior, MaternPrior):
        return matern_jvp(h, dh, prior, bins)
    nb = prior.n_bins
    (th_fl, th_sl, th_fx, th_as), (s_fl, s_sl, s_fx, s_as), xi1, xi2 = _thetas(h, prior)
    d_fl, d_sl, d_fx, d_as, dxi1, dxi2 = _split(dh, nb)
    f = forward(h, prior, bins)
    a, S, c = f["a"], f["S"], f["c"]
    dth_fl = th_fl * s_fl * d_fl
    dth_sl = s_sl * d_sl
    dth_fx = th_fx * s_fx * d_fx
    dth_as = th_as * s_as * d_as
    l = bins.centres
    dx = np.zeros(nb)
    dy = np.zeros(nb)
    for i in range(1, nb):
        d = l[i] - l[i - 1]
        dx[i] = dx[i - 1] + dth_fx * np.sqrt(d) * xi1[i - 1] + th_fx * np.sqrt(d) * dxi1[i - 1]
        dc = d * dth_as / (2.0 * c[i])
        dy[i] = (dy[i - 1] + d * (dx[i - 1] + dx[i]) / 2.0
                 + (dth_fx * c[i] + th_fx * dc) * xi2[i - 1] + th_fx * c[i] * dxi2[i - 1])
    dtau = dth_sl * (l - l[0]) + dy
    da = a * dtau / 2.0
    dS = np.sum(bins.counts * 2.0 * a * da)
    rs = 1.0 / np.sqrt(S)
    return dth_fl * a * rs + th_fl * da * rs - th_fl * a * dS * rs ** 3 / 2.0


def vjp(h, gA, prior, bins):
    """Reverse-mode derivative: the hyper-latent cotangent for cotangent ``gA``."""
    if isinstance(prior, MaternPrior):
        return matern_vjp(h, gA, prior, bins)
    nb = prior.n_bins
    (th_fl, th_sl, th_fx, th_as), (s_fl, s_sl, s_fx, s_as), xi1, xi2 = _thetas(h, prior)
    gA = np.asarray(gA, dtype=np.float64)
    f = forward(h, prior, bins)
    a, S, c = f["a"], f["S"], f["c"]
    rs = 1.0 / np.sqrt(S)
    ga_dot = np.sum(gA * a)
    g_thfl = ga_dot * rs
    # A_b = th_fl a_b S^-1/2 with S = sum n a^2
    g_a = th_fl * rs * gA - th_fl * rs ** 3 * bins.counts * a * ga_dot
    g_tau = g_a * a / 2.0
    l = bins.centres
    g_thsl = np.sum(g_tau * (l - l[0]))
    # total adjoint of y_i: y_i feeds tau_i and every later y_j
    y_hat = np.zeros(nb)
    acc = 0.0
    for i in range(nb - 1, -1, -1):
        acc += g_tau[i]
        y_hat[i] = acc
    g_xi2 = np.zeros(nb - 1)
    g_thfx = 0.0
    g_thas = 0.0
    x_dir = np.zeros(nb)
    for i in range(1, nb):
        d = l[i] - l[i - 1]
        x_dir[i - 1] += y_hat[i] * d / 2.0
        x_dir[i] += y_hat[i] * d / 2.0
        g_xi2[i - 1] = y_hat[i] * th_fx * c[i]
        g_thfx += y_hat[i] * c[i] * xi2[i - 1]
        g_c = y_hat[i] * th_fx * xi2[i - 1]
        g_thas += g_c * d / (2.0 * c[i])
    x_hat = np.zeros(nb)
    acc = 0.0
    for i in range(nb - 1, -1, -1):
        acc += x_dir[i]
        x_hat[i] = acc
    g_xi1 = np.zeros(nb - 1)
    for i in range(1, nb):
        d = l[i] - l[i - 1]
        g_xi1[i - 1] = x_hat[i] * th_fx * np.sqrt(d)
        g_thfx += x_hat[i] * np.sqrt(d) * xi1[i - 1]
    out = np.zeros(4 + 2 * (nb - 1))
    out[0] = g_thfl * th_fl * s_fl
    out[1] = g_thsl * s_sl
    out[2] = g_thfx * th_fx * s_fx
    out[3] = g_thas * th_as * s_as
    out[4:4 + nb - 1] = g_xi1
    out[4 + nb - 1:] = g_xi2
    return out


# ---------------------------------------------------------------- Matern


def _matern_thetas(h, prior):
    h = np.asarray(h, dtype=np.float64)
    assert h.shape == (3,)
    mu_sc, s_sc = lognormal_params(*prior.scale)
    mu_ct, s_ct = lognormal_params(*prior.cutoff)
    th_sc = np.exp(mu_sc + s_sc * h[0])
    th_ct = np.exp(mu_ct + s_ct * h[1])
    th_al = prior.loglogslope[0] + prior.loglogslope[1] * h[2]
    return (th_sc, th_ct, th_al), (s_sc, s_ct, prior.loglogslope[1])


def matern_forward(h, prior, bins):
    """Matern amplitude per bin and its intermediates (see the module text)."""
    (th_sc, th_ct, th_al), _ = _matern_thetas(h, prior)
    k = np.exp(bins.centres)
    L = np.log1p((k / th_ct) ** 2)          # ln(1 + (k / cutoff)^2)
    a = np.exp(th_al * L / 4.0)
    S = np.sum(bins.counts * a * a)
    A = th_sc * a / np.sqrt(S)
    return dict(A=A, a=a, S=S, L=L, k=k, theta=(th_sc, th_ct, th_al))


def matern_jvp(h, dh, prior, bins):
    (th_sc, th_ct, th_al), (s_sc, s_ct, s_al) = _matern_thetas(h, prior)
    dh = np.asarray(dh, dtype=np.float64)
    f = matern_forward(h, prior, bins)
    a, S, L, k = f["a"], f["S"], f["L"], f["k"]
    dsc = th_sc * s_sc * dh[0]
    dct = th_ct * s_ct * dh[1]
    dal = s_al * dh[2]
    r = (k / th_ct) ** 2
    # d ln a = dal L / 4 + (th_al / 4) d ln(1 + r),  d ln(1 + r) = -2 r / (1 + r) dct / th_ct
    dlna = dal * L / 4.0 - (th_al / 2.0) * r / (1.0 + r) * dct / th_ct
    da = a * dlna
    dS = np.sum(bins.counts * 2.0 * a * da)
    rs = 1.0 / np.sqrt(S)
    return dsc * a * rs + th_sc * da * rs - th_sc * a * dS * rs ** 3 / 2.0


def matern_vjp(h, gA, prior, bins):
    (th_sc, th_ct, th_al), (s_sc, s_ct, s_al) = _matern_thetas(h, prior)
    gA = np.asarray(gA, dtype=np.float64)
    f = matern_forward(h, prior, bins)
    a, S, L, k = f["a"], f["S"], f["L"], f["k"]
    rs = 1.0 / np.sqrt(S)
    ga_dot = np.sum(gA * a)
    g_sc = ga_dot * rs
    g_a = th_sc * rs * gA - th_sc * rs ** 3 * bins.counts * a * ga_dot
    g_lna = g_a * a
    r = (k / th_ct) ** 2
    g_al = np.sum(g_lna * L / 4.0)
    g_ct = np.sum(g_lna * (-(th_al / 2.0) * r / (1.0 + r) / th_ct))
    return np.array([g_sc * th_sc * s_sc, g_ct * th_ct * s_ct, g_al * s_al])
