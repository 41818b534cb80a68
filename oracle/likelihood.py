"""Fisher weights of the likelihoods at an expansion point (oracle; test infrastructure only).

Sec. "Performance": the Fisher metric of the likelihood is J^T N^-1 J with
N^-1 the Fisher metric of the likelihood in data space.  With a response
s = R(cf) applied pointwise, J^T N^-1 J = J_cf^T diag(w) J_cf where

* Gaussian, noise std sigma, observed-pixel mask m:  N^-1 = m / sigma^2,
  so w = m * R'(cf_p)^2 / sigma^2  (R = exp: w = m s_p^2 / sigma^2;
  R = identity: w = m / sigma^2);
* Poisson with rate lambda = scale * exp(cf) (Sec. "Building Up Complex Models":
  ``jft.Poissonian(data).amend(forward)`` with forward = exp(cf); the benchmark
  multiplies by 10): N^-1 = 1/lambda, d lambda/d cf = lambda, so w = lambda_p.

The data never enter M, only the KL gradient.
"""
import numpy as np


def gaussian_weight(cf_p, sigma, mask=None, response="exp"):
    cf_p = np.asarray(cf_p, dtype=np.float64)
    m = np.ones_like(cf_p) if mask is None else np.asarray(mask, dtype=np.float64)
    if response == "exp":
        s = np.exp(cf_p)
        return m * s * s / (sigma * sigma)
    if response == "identity":
        return m / (sigma * sigma)
    raise ValueError(response)


def poisson_weight(cf_p, scale=10.0):
    return scale * np.exp(np.asarray(cf_p, dtype=np.float64))
