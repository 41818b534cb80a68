"""Metric-vector product and MGVI right-hand side (oracle; test infrastructure only).

Sec. "Performance": M_p := F_p + 1 with F_p = J^T N^-1 J, J the Jacobian of the
forward model at p.  With the weight w of ``oracle.likelihood`` (which already
holds the response Jacobian squared) and J = d cf / d xi:

    M_p v = v + J^T (w * J v).

Sec. "Variational Inference": MGVI draws samples around p from N(p, M_p^-1).
A right-hand side with covariance M_p is b = xi' + J^T (sqrt(w) * eta) with
xi' ~ N(0, I) in latent space and eta ~ N(0, I) in data space; the sample is
p +/- M_p^-1 b (antithetic pair).
"""
import numpy as np


def metric_apply(model, xi_p, w, v):
    jv = model.jvp(xi_p, v)
    return np.asarray(v, dtype=np.float64) + model.vjp(xi_p, w * jv)


def mgvi_rhs(model, xi_p, w, xi_prime, eta):
    eta = np.asarray(eta, dtype=np.float64).reshape(model.shape)
    return np.asarray(xi_prime, dtype=np.float64) + model.vjp(xi_p, np.sqrt(w) * eta)


def dense_metric(model, xi_p, w):
    """M assembled column by column (tiny problems only)."""
    n = model.latent_size
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = metric_apply(model, xi_p, w, e)
    return M
