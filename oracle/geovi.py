"""geoVI nonlinear sample update (oracle; test infrastructure only).

Sec. "Variational Inference": geoVI, the successor of MGVI, draws samples
around an expansion point p whose shape follows the posterior's geometry; the
example updates the linear samples nonlinearly with a Newton minimiser "SN"
(``nonlinearly_update_kwargs``: xtol, maxiter = 5).  The paper gives no
formulas; the reading used throughout this project:

* t is the likelihood's standardising transform in data space, the map under
  which the likelihood's Fisher metric is the identity:
      Gaussian (std sigma, mask m, response R):  t(cf) = sqrt(m) R(cf) / sigma,
      Poisson (rate lambda = scale exp(cf)):     t(cf) = 2 sqrt(lambda),
  so that with J_p the Jacobian of xi -> t(cf(xi)) at p, J_p^T J_p is the
  likelihood part of the MGVI metric M_p = I + J_p^T J_p.
* The sample residual delta solves the coordinate equation
      F(delta) = delta + J_p^T [t(cf(p + delta)) - t(cf(p))] - b = 0,
  whose linearisation at delta = 0 is M_p delta = b: the linear MGVI residual
  delta_0 = M_p^-1 b (b = xi' + J_p^T eta, Cov b = M_p) is the starting point,
  and for a linear t it solves F exactly.
* Newton iterations with M_p as the Jacobian of F:
      delta <- delta - M_p^-1 F(delta)  (CG to cg_rtol),
  at most maxiter of them, stopping once mean_i |step_i| <= xtol.
  The antithetic partner uses -b.
"""
import numpy as np

from .cg import cg
from .metric import metric_apply


def transform(lik, cf):
    """t(cf) and dt/dcf, pointwise.  lik: ("poisson", scale) or ("gauss", sigma,
    mask or None, response)."""
    cf = np.asarray(cf, dtype=np.float64)
    if lik[0] == "poisson":
        lam = lik[1] * np.exp(cf)
        return 2.0 * np.sqrt(lam), np.sqrt(lam)
    sigma, mask, resp = lik[1], lik[2], lik[3]
    m = np.ones_like(cf) if mask is None else np.asarray(mask, dtype=np.float64).reshape(cf.shape)
    s = np.exp(cf) if resp == "exp" else cf
    ds = s if resp == "exp" else np.ones_like(cf)
    return np.sqrt(m) * s / sigma, np.sqrt(m) * ds / sigma


def coordinate_residual(model, lik, p, b, delta):
    """F(delta) = delta + J_p^T [t(p + delta) - t(p)] - b."""
    tp, dtp = transform(lik, model.forward(p))
    tq, _ = transform(lik, model.forward(np.asarray(p) + delta))
    return np.asarray(delta, dtype=np.float64) + model.vjp(p, dtp * (tq - tp)) - np.asarray(b, dtype=np.float64)


def nonlinear_update(model, lik, p, w, b, delta0, xtol=1e-4, maxiter=5, cg_rtol=1e-6, cg_maxiter=500):
    """Newton iterations on F from delta0; w are the Fisher weights at p (the
    metric's).  Returns (delta, iterations, [mean |step|])."""
    mv = lambda v: metric_apply(model, p, w, v)
    delta = np.asarray(delta0, dtype=np.float64).copy()
    steps = []
    it = 0
    while it < maxiter:
        F = coordinate_residual(model, lik, p, b, delta)
        step, _, _ = cg(mv, F, rtol=cg_rtol, maxiter=cg_maxiter)
        delta = delta - step
        it += 1
        steps.append(float(np.mean(np.abs(step))))
        if steps[-1] <= xtol:
            break
    return delta, it, steps
