"""Conjugate gradients for the linear sample draw (oracle; test infrastructure only).

Sec. "Variational Inference": the linear part of a sample draw solves M_p x = b by
conjugate gradients (``draw_linear_kwargs`` / ``cg_kwargs``, ``maxiter=100``).
Reading of the stopping rule: stop before an iteration once the recursive
residual satisfies ||r_k|| <= rtol ||b||, or after ``maxiter`` iterations
(rtol = 0 runs exactly maxiter iterations).  Textbook Hestenes-Stiefel:

    x_0 = 0, r_0 = b, p_0 = r_0
    alpha = (r.r) / (p.Mp);  x += alpha p;  r -= alpha Mp
    beta = (r'.r') / (r.r);  p = r' + beta p
"""
import numpy as np


def cg(matvec, b, rtol=0.0, maxiter=100, callback=None):
    """Return (x, iterations, relres) with relres = ||r_k|| / ||b||."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bn = np.sqrt(float(b @ b))
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxiter:
        if np.sqrt(rr) <= rtol * bn:
            break
        q = matvec(p)
        alpha = rr / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        it += 1
        if callback is not None:
            callback(it, x)
    return x, it, np.sqrt(rr) / bn
