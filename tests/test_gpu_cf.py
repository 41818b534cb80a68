"""GPU parity of the correlated field through the C ABI: cf_forward, cf_jvp and
cf_vjp against the FP64 oracle on the same seeded inputs.

Tolerance (rel_max = max |gpu - oracle| / max |oracle|, per latent block):
FP64 plans 1e-12; FP32 plans 1e-5 (the FP32 transforms carry a relative error
of order eps_32 * log2 N ~ 1e-6).  Sizes span several sweeps, odd batches (the
1-D sweep pairs samples), the smallest grids, non-square and mixed-length axes.
"""
import numpy as np
import pytest
import torch

import synth
from helpers import blocks_rel, cf_pair, field_to_dev, host, rel_max, rounded, to_dev

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}

CASES = [
    ((256,), "matern", "f64", 256),
    ((4096,), "power", "f64", 256),
    ((8,), "matern", "f64", 256),
    ((4, 4), "power", "f64", 8),
    ((16, 32), "power", "f64", 256),
    ((64, 8), "matern", "f64", 256),
    ((8, 16, 8), "power", "f64", 32),
    ((4, 8, 16), "matern", "f64", 256),
    ((256,), "power", "f32", 256),
    ((64, 64), "power", "f32", 256),
    ((32, 16, 64), "power", "f32", 256),
    ((4096, 8), "matern", "f32", 256),
    # lines of 512 / 1024 / 2048 points along either axis (each FFT exchange
    # has its own shared-memory layout from 256 points on)
    ((2048,), "power", "f32", 256),
    ((16, 2048), "power", "f32", 256),
    ((2048, 16), "power", "f32", 256),
    ((8, 1024), "matern", "f32", 256),
    ((512, 8), "power", "f32", 256),
    # the parametric Matern amplitude (three hyper-parameters on the log-|k| bins)
    ((256,), "matern_model", "f64", 64),
    ((32, 16), "matern_model", "f64", 256),
    ((8, 16, 32), "matern_model", "f64", 32),
    ((4096,), "matern_model", "f32", 256),
    ((128, 256), "matern_model", "f32", 256),
    ((32, 32, 64), "matern_model", "f32", 256),
]


def _inputs(om, B, dtype, seed):
    g = np.random.default_rng(seed)
    xi = rounded(g.standard_normal((B, om.latent_size)), dtype)
    v = rounded(g.standard_normal((B, om.latent_size)), dtype)
    ct = rounded(g.standard_normal((B, om.n_field)), dtype)
    return xi, v, ct


@pytest.mark.parametrize("shape,kind,dtype,nb", CASES)
def test_cf_forward_jvp_vjp(shape, kind, dtype, nb):
    plan, om = cf_pair(shape, kind, dtype, n_bins=nb)
    B = 3
    xi, v, ct = _inputs(om, B, dtype, 100 + len(shape))
    s = host(plan.forward(to_dev(plan, xi)))
    jv = host(plan.jvp(to_dev(plan, xi), to_dev(plan, v)))
    g = host(plan.vjp(to_dev(plan, xi), field_to_dev(plan, ct)), om.latent_size)
    torch.cuda.synchronize()
    for b in range(B):
        assert rel_max(s[b], om.forward(xi[b]).ravel()) <= TOL[dtype]
        assert rel_max(jv[b], om.jvp(xi[b], v[b]).ravel()) <= TOL[dtype]
        assert blocks_rel(g[b], om.vjp(xi[b], ct[b]), om.n_field) <= TOL[dtype]


def test_cf_full_size_512():
    """2-D 512^2 power model, FP32, batch 2 (the benchmark grid)."""
    plan, om = cf_pair((512, 512), "power", "f32")
    xi, v, ct = _inputs(om, 2, "f32", 7)
    s = host(plan.forward(to_dev(plan, xi)))
    jv = host(plan.jvp(to_dev(plan, xi), to_dev(plan, v)))
    g = host(plan.vjp(to_dev(plan, xi), field_to_dev(plan, ct)), om.latent_size)
    for b in range(2):
        assert rel_max(s[b], om.forward(xi[b]).ravel()) <= 1e-5
        assert rel_max(jv[b], om.jvp(xi[b], v[b]).ravel()) <= 1e-5
        assert blocks_rel(g[b], om.vjp(xi[b], ct[b]), om.n_field) <= 1e-5


def test_batch_zero_and_layout():
    plan, om = cf_pair((16, 16), "power", "f32", n_bins=16)
    assert plan.latent_size == 256 + 4 + 2 * 15
    assert plan.stride % 64 == 0 and plan.stride >= plan.latent_size
    z = torch.zeros(0, plan.stride, device="cuda:0")
    assert plan.forward(z).shape == (0, 256)


def test_cf_sample_covariance_matches_spectrum():
    """Empirical covariance of GPU draws (1-D fixed spectrum) against the closed
    form sum_k A_k^2 cos(2 pi k d / N) (a property that holds at any size)."""
    N = 256
    plan, om = cf_pair((N,), "matern", "f64")
    n = 20000
    xi = torch.randn(n, N, dtype=torch.float64, device="cuda:0", generator=torch.Generator("cuda:0").manual_seed(3))
    s = plan.forward(plan.pad(xi))
    C = (s.T @ s / n).cpu().numpy()
    A = om.fixed.ravel()
    k = np.arange(N)
    for d in [0, 1, 4, 16, 64, 128]:
        ref = np.sum(A ** 2 * np.cos(2 * np.pi * k * d / N))
        sd = np.sqrt((1.0 + ref ** 2) / n)
        est = np.mean([C[i, (i + d) % N] for i in range(0, N, 17)])
        assert abs(est - ref) <= 5 * sd
