"""Correlated-field model, its JVP and VJP (oracle; test infrastructure only).

Sec. "Gaussian Processes": s = FT o sqrt(P) o xi with standard-normal xi
(standardization, Sec. "Core Components").  Readings:

* FT is the unnormalised multi-dimensional Hartley transform H (``oracle.dht``).
* The field excitation xi_field has one entry per harmonic pixel; its zero mode
  carries the offset: A_full[0] = offset_std, A_full[k] = A[bin(k)] for k != 0,
  and cf(xi) = offset_mean + H(A_full * xi_field) (cas(0) = 1, so the zero mode
  adds a constant in position space).
* Two amplitude kinds:
  - "model": the non-parametric power model of ``oracle.amplitude``; the latent
    vector is [xi_field (N), hyper (4 + 2 (n_bins - 1))];
  - "fixed": a given per-pixel A_full (no hyper-parameters); the latent vector is
    xi_field alone.  ``matern_fixed_amplitude`` builds the 1-D benchmark
    spectrum A(k) = (1 + (|k|/k0)^2)^-gamma normalised to a total variance.

The JVP at xi_p in direction v and the VJP with cotangent g are the plain chain
rule of this definition:
    d cf = H(A_full * v_field + dA_full * xi_p_field),
    g_field = A_full * H(g),   g_A[b] = sum_{k in bin b} xi_p_field[k] H(g)[k],
then g_hyper = VJP of the amplitude model applied to g_A.
"""
import numpy as np

from . import amplitude as amp_mod
from .dht import dht
from .grid import LogBins, k_norm


def matern_fixed_amplitude(shape, spacing, k0=8.0, gamma=1.5, variance=1.0, zero_mode=0.0):
    """Per-pixel A_full = (1 + (|k|/k0)^2)^-gamma with sum_{k != 0} A^2 = variance."""
    kn = k_norm(shape, spacing)
    a = (1.0 + (kn / k0) ** 2) ** (-gamma)
    nz = kn > 0
    a = a * np.sqrt(variance / np.sum(a[nz] ** 2))
    a[~nz] = zero_mode
    return a


class CFModel:
    def __init__(self, shape, spacing, prior=None, fixed_amp=None, offset_mean=0.0):
        self.shape = tuple(int(s) for s in shape)
        self.spacing = tuple(float(s) for s in spacing)
        self.n_field = int(np.prod(self.shape))
        if (prior is None) == (fixed_amp is None):
            raise ValueError("give exactly one of prior / fixed_amp")
        self.prior = prior
        if prior is not None:
            self.bins = LogBins(self.shape, self.spacing, prior.n_bins)
            self.n_hyper = prior.n_hyper
            self.offset_mean = prior.offset_mean
        else:
            self.fixed = np.asarray(fixed_amp, dtype=np.float64).reshape(self.shape)
            self.n_hyper = 0
            self.offset_mean = float(offset_mean)

    @property
    def latent_size(self):
        return self.n_field + self.n_hyper

    def split(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        assert xi.shape == (self.latent_size,)
        return xi[:self.n_field].reshape(self.shape), xi[self.n_field:]

    def _full(self, per_bin, zero):
        out = np.empty(self.shape)
        nz = self.bins.index >= 0
        out[nz] = per_bin[self.bins.index[nz]]
        out[~nz] = zero
        return out

    def a_full(self, hyper):
        if self.prior is None:
            return self.fixed
        A = amp_mod.amplitude(hyper, self.prior, self.bins)
        return self._full(A, self.prior.offset_std)

    def da_full(self, hyper, dhyper):
        if self.prior is None:
            return np.zeros(self.shape)
        dA = amp_mod.jvp(hyper, dhyper, self.prior, self.bins)
        return self._full(dA, 0.0)

    def forward(self, xi):
        f, h = self.split(xi)
        return self.offset_mean + dht(self.a_full(h) * f)

    def jvp(self, xi_p, v):
        fp, hp = self.split(xi_p)
        vf, vh = self.split(v)
        u = self.a_full(hp) * vf + self.da_full(hp, vh) * fp
        return dht(u)

    def vjp(self, xi_p, g):
        fp, hp = self.split(xi_p)
        r = dht(np.asarray(g, dtype=np.float64).reshape(self.shape))
        out = np.zeros(self.latent_size)
        out[:self.n_field] = (self.a_full(hp) * r).ravel()
        if self.prior is not None:
            nz = self.bins.index >= 0
            gA = np.bincount(self.bins.index[nz], weights=(fp * r)[nz],
                             minlength=self.prior.n_bins)
            out[self.n_field:] = amp_mod.vjp(hp, gA, self.prior, self.bins)
        return out
