"""KL minimisation of MGVI by Newton-CG (oracle; test infrastructure only).

Sec. "Variational Inference": MGVI alternates between drawing samples around an
expansion point and minimising the Kullback-Leibler divergence for the shape
those samples define; the KL minimiser of the example is "M", a Newton-CG
(``kl_kwargs``: ``xtol``, ``maxiter=35``).  The paper gives no formulas; the
reading used throughout this project:

* Samples xi_s = xi_bar + delta_s, s = 1..S, with the residual samples delta_s
  (antithetic pairs +-delta from the linear draw) held fixed while xi_bar moves.
* Energy (the sample estimate of the KL up to constants), with the
  standardised prior of Sec. "Core Components":
      E(xi_bar) = (1/S) sum_s [ NLL(d | cf(xi_s)) + |xi_s|^2 / 2 ],
  NLL dropping data-only constants:
      Poisson, rate lambda = scale exp(cf):  sum_x lambda_x - d_x ln lambda_x;
      Gaussian, response R, mask m, std sigma:  sum_x m_x (d_x - R(cf_x))^2 / (2 sigma^2).
* Gradient: grad E = (1/S) sum_s [ xi_s + J_s^T dNLL/dcf(xi_s) ] with
      Poisson dNLL/dcf = lambda - d;  Gaussian dNLL/dcf = -m (d - R(cf)) R'(cf) / sigma^2.
* Curvature of the Newton step: the sample-averaged metric
      Mbar = I + (1/S) sum_s J_s^T W_s J_s,
  W_s the Fisher weights at xi_s (``oracle.likelihood``).
* Newton-CG iteration: D = -Mbar^-1 grad E by CG (x_0 = 0; stop at relative
  recursive residual cg_rtol or cg_maxiter iterations); backtracking line
  search: alpha = 1, halved while E(xi_bar + alpha D) > E(xi_bar), at most 30
  times (no decrease: the step is zero and the minimisation stops);
  xi_bar += alpha D.  Stop once mean_i |alpha D_i| <= xtol (the paper scales
  its absolute tolerance by the number of latent entries) or after maxiter
  iterations.
"""
import numpy as np

from .cg import cg
from .likelihood import gaussian_weight, poisson_weight


class KLProblem:
    """The KL energy of one correlated-field model and likelihood for fixed
    residual samples.  lik: ("poisson", scale) or ("gauss", sigma, mask or
    None, response "exp" / "identity")."""

    def __init__(self, model, lik, data, deltas):
        self.model = model
        self.lik = lik
        self.data = np.asarray(data, dtype=np.float64).reshape(model.shape)
        self.deltas = [np.asarray(d, dtype=np.float64) for d in deltas]
        self.S = len(self.deltas)

    # likelihood pieces, pointwise in cf ------------------------------------
    def nll(self, cf):
        d = self.data
        if self.lik[0] == "poisson":
            lam = self.lik[1] * np.exp(cf)
            return float(np.sum(lam - d * np.log(lam)))
        sigma, mask, resp = self.lik[1], self.lik[2], self.lik[3]
        m = np.ones_like(cf) if mask is None else np.asarray(mask, dtype=np.float64).reshape(cf.shape)
        s = np.exp(cf) if resp == "exp" else cf
        return float(np.sum(m * (d - s) ** 2) / (2 * sigma * sigma))

    def dnll(self, cf):
        d = self.data
        if self.lik[0] == "poisson":
            return self.lik[1] * np.exp(cf) - d
        sigma, mask, resp = self.lik[1], self.lik[2], self.lik[3]
        m = np.ones_like(cf) if mask is None else np.asarray(mask, dtype=np.float64).reshape(cf.shape)
        s = np.exp(cf) if resp == "exp" else cf
        ds = s if resp == "exp" else np.ones_like(cf)
        return -m * (d - s) * ds / (sigma * sigma)

    def weight(self, cf):
        if self.lik[0] == "poisson":
            return poisson_weight(cf, self.lik[1])
        mask = self.lik[2]
        if mask is not None:
            mask = np.asarray(mask, dtype=np.float64).reshape(cf.shape)
        return gaussian_weight(cf, self.lik[1], mask=mask, response=self.lik[3])

    # KL ---------------------------------------------------------------------
    def points(self, xi_bar):
        return [np.asarray(xi_bar, dtype=np.float64) + d for d in self.deltas]

    def energy(self, xi_bar):
        e = 0.0
        for xs in self.points(xi_bar):
            e += self.nll(self.model.forward(xs)) + 0.5 * float(xs @ xs)
        return e / self.S

    def gradient(self, xi_bar):
        g = np.zeros(self.model.latent_size)
        for xs in self.points(xi_bar):
            g += xs + self.model.vjp(xs, self.dnll(self.model.forward(xs)))
        return g / self.S

    def metric_apply(self, xi_bar, v):
        v = np.asarray(v, dtype=np.float64)
        out = np.zeros_like(v)
        for xs in self.points(xi_bar):
            w = self.weight(self.model.forward(xs))
            out += self.model.vjp(xs, w * self.model.jvp(xs, v))
        return v + out / self.S

    def newton_step(self, xi_bar, cg_rtol=1e-3, cg_maxiter=200):
        """One Newton-CG iteration; returns (new xi_bar, alpha D, energy)."""
        xi_bar = np.asarray(xi_bar, dtype=np.float64)
        g = self.gradient(xi_bar)
        D, _, _ = cg(lambda p: self.metric_apply(xi_bar, p), -g, rtol=cg_rtol, maxiter=cg_maxiter)
        e0 = self.energy(xi_bar)
        alpha = 1.0
        for _ in range(31):
            e1 = self.energy(xi_bar + alpha * D)
            if e1 <= e0:
                return xi_bar + alpha * D, alpha * D, e1
            alpha *= 0.5
        return xi_bar, np.zeros_like(D), e0

    def minimize(self, xi_bar, xtol=1e-4, maxiter=35, cg_rtol=1e-3, cg_maxiter=200):
        """Newton-CG to mean |step| <= xtol; returns (xi_bar, iterations, energies)."""
        x = np.asarray(xi_bar, dtype=np.float64)
        energies = [self.energy(x)]
        it = 0
        while it < maxiter:
            x, step, e = self.newton_step(x, cg_rtol, cg_maxiter)
            energies.append(e)
            it += 1
            if np.mean(np.abs(step)) <= xtol:
                break
        return x, it, energies
