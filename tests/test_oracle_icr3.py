"""Pins of the oracle's 3-D charted refinement (CPU only).

Pinned by: the level-0 covariance; one refinement from an exact level 0
reproduces the kernel on every child block and its 3x3x3 neighbourhood
(clamped radial and polar windows, periodic azimuth, child order 4a + 2b + c),
with positions and the Matern-3/2 kernel written out here; a voxel outside the
neighbourhood breaks that identity; R and D against the joint precision
matrix; linearity, the adjoint identity and central differences.
"""
import numpy as np
import pytest

from oracle.icr3 import ICRChart3D


def _pos(n0, level, i, j, k):
    n = n0 * 2 ** level
    u, v, t = (i + 0.5) / n, (j + 0.5) / n, (k + 0.5) / n
    r = 0.1 * 10.0 ** u
    th, ph = np.pi * v, 2 * np.pi * t
    return np.array([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)])


def _k(pa, pb, rho):
    d = np.linalg.norm(pa - pb)
    return (1.0 + np.sqrt(3.0) * d / rho) * np.exp(-np.sqrt(3.0) * d / rho)


def _dense(c):
    n = c.latent_size
    cols = [c.forward(np.eye(n)[j], return_levels=True) for j in range(n)]
    return [np.stack([col[l].ravel() for col in cols], axis=1) for l in range(c.n_levels + 1)]


def test_icr3_level0_covariance():
    c = ICRChart3D(n0=3, n_levels=1, rho=0.3)
    L = c.L0()
    idx = [(i, j, k) for i in range(3) for j in range(3) for k in range(3)]
    K = np.array([[_k(_pos(3, 0, *a), _pos(3, 0, *b), 0.3) for b in idx] for a in idx])
    np.testing.assert_allclose(L @ L.T, K, atol=1e-12)


@pytest.mark.parametrize("n0,rho", [(4, 0.5), (4, 0.25), (5, 0.4)])
def test_icr3_one_refinement_reproduces_kernel(n0, rho):
    c = ICRChart3D(n0=n0, n_levels=1, rho=rho)
    L0, L1 = _dense(c)
    C10, C11 = L1 @ L0.T, L1 @ L1.T
    n1 = 2 * n0
    flat1 = lambda i, j, k: (i * n1 + j) * n1 + k
    flat0 = lambda i, j, k: (i * n0 + j) * n0 + k
    worst = 0.0
    for i in range(n0):
        wi = min(max(i - 1, 0), n0 - 3)
        for j in range(n0):
            wj = min(max(j - 1, 0), n0 - 3)
            for k in (0, 1, n0 - 1):
                nbh = [(wi + a, wj + b, (k + d) % n0) for a in range(3) for b in range(3) for d in (-1, 0, 1)]
                kids = [(2 * i + a, 2 * j + b, 2 * k + e) for a in range(2) for b in range(2) for e in range(2)]
                for f in kids:
                    pf = _pos(n0, 1, *f)
                    for q in nbh:
                        worst = max(worst, abs(C10[flat1(*f), flat0(*q)] - _k(pf, _pos(n0, 0, *q), rho)))
                    for g in kids:
                        worst = max(worst, abs(C11[flat1(*f), flat1(*g)] - _k(pf, _pos(n0, 1, *g), rho)))
    assert worst <= 1e-11, worst


def test_icr3_outside_neighbour_breaks_identity():
    n0, rho = 5, 0.5
    c = ICRChart3D(n0=n0, n_levels=1, rho=rho)
    L0, L1 = _dense(c)
    C10 = L1 @ L0.T
    i, j, k = 2, 2, 2                           # interior: windows 1..3
    f = (2 * i, 2 * j, 2 * k)
    q = (i, j + 2, k)                           # polar row 4, outside the window
    n1 = 2 * n0
    got = C10[(f[0] * n1 + f[1]) * n1 + f[2], (q[0] * n0 + q[1]) * n0 + q[2]]
    assert abs(got - _k(_pos(n0, 1, *f), _pos(n0, 0, *q), rho)) > 1e-6


@pytest.mark.parametrize("i,j", [(0, 0), (1, 2), (3, 3)])
def test_icr3_matrices_match_joint_precision(i, j):
    c = ICRChart3D(n0=4, n_levels=1, rho=0.4)
    R, LD = c.matrices(0)
    pc, pf = c.coarse_fine_points(0, i, j)
    pts = np.concatenate([pf, pc])
    K = np.array([[_k(a, b, 0.4) for b in pts] for a in pts])
    Lam = np.linalg.inv(K)
    D = np.linalg.inv(Lam[:8, :8])
    np.testing.assert_allclose(R[i, j], -D @ Lam[:8, 8:], atol=1e-7)
    np.testing.assert_allclose(LD[i, j] @ LD[i, j].T, D, atol=1e-8)


def test_icr3_linearity_adjoint_fd():
    c = ICRChart3D(n0=3, n_levels=2, rho=0.3)
    g = np.random.default_rng(0)
    a, b = g.standard_normal((2, c.latent_size))
    np.testing.assert_allclose(c.forward(0.3 * a - 1.2 * b), 0.3 * c.forward(a) - 1.2 * c.forward(b), atol=1e-12)
    ct = g.standard_normal(c.forward(a).shape)
    lhs = np.sum(c.forward(a) * ct)
    assert abs(lhs - a @ c.vjp(ct)) <= 1e-12 * abs(lhs)
    h = 1e-3
    np.testing.assert_allclose((c.forward(a + h * b) - c.forward(a - h * b)) / (2 * h), c.jvp(b), atol=1e-10)
    Mu = c.metric_apply(a)
    assert abs(Mu @ b - a @ c.metric_apply(b)) <= 1e-11 * np.linalg.norm(Mu) * np.linalg.norm(b)
