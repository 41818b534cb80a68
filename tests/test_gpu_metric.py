"""GPU parity of the metric M_p = J^T N^-1 J + 1, the MGVI right-hand side and
batched CG through the C ABI, against the FP64 oracle.

Tolerances: metric products and right-hand sides rel_max <= 1e-12 (FP64) and
<= 1e-5 (FP32).  CG iterates under rounding: see test_cg_config1_per_iteration
(iterates compared while CG is insensitive to one-ulp perturbations, energy-norm
optimality afterwards); converged solves are judged by the oracle's FP64 true
residual ||b - M x|| / ||b|| and, in FP64, by the distance to the oracle's
solution.
"""
import numpy as np
import pytest
import torch

import synth
from helpers import DEV, blocks_rel, cf_pair, host, rel_l2, rel_max, rounded, to_dev
from oracle.cg import cg as ocg
from oracle.likelihood import gaussian_weight, poisson_weight
from oracle.metric import metric_apply as ometric
from oracle.metric import mgvi_rhs as orhs

pytestmark = pytest.mark.gpu


def _lik(nre, kind, om, mask=None, sigma=0.1):
    if kind == "poisson":
        return nre.Likelihood("poisson", scale=10.0), lambda cf: poisson_weight(cf, 10.0)
    return (nre.Likelihood("gauss", sigma=sigma, mask=mask),
            lambda cf: gaussian_weight(cf, sigma, mask=None if mask is None else mask.reshape(cf.shape)))


def _setup(shape, kind, dtype, lik, seed=1, max_batch=4, n_bins=256, mask=None, sigma=0.1, xi_scale=1.0):
    import paper_2402_16683_gb300 as nre
    plan, om = cf_pair(shape, kind, dtype, n_bins=n_bins)
    xi_p = rounded(xi_scale * synth.normal(seed, om.latent_size), dtype)
    L, wfun = _lik(nre, lik, om, mask=mask, sigma=sigma)
    M = nre.Metric(plan, L, to_dev(plan, xi_p)[0], max_batch=max_batch)
    w = wfun(om.forward(xi_p))
    return plan, om, M, xi_p, w


def lanczos_kappa(om, xi_p, w, b, iters):
    """Condition-number estimate from the CG (Lanczos) coefficients of the oracle."""
    alphas, betas = [], []
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    for _ in range(iters):
        q = ometric(om, xi_p, w, p)
        a = rr / (p @ q)
        r = r - a * q
        rn = r @ r
        be = rn / rr
        alphas.append(a)
        betas.append(be)
        p = r + be * p
        rr = rn
    k = len(alphas)
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    ev = np.linalg.eigvalsh(T)
    return ev[-1] / ev[0]


@pytest.mark.parametrize("shape,kind,dtype,lik", [
    ((256,), "matern", "f64", "gauss"),
    ((256,), "power", "f64", "poisson"),
    ((32, 64), "power", "f64", "poisson"),
    ((16, 8, 32), "power", "f64", "gauss"),
    # FP64 rows of 256 points: the bulk-copy row staging of 2-D and 3-D orbits
    ((128, 256), "power", "f64", "poisson"),
    ((4, 8, 256), "power", "f64", "gauss"),
    ((512, 512), "power", "f32", "poisson"),
    # 256-point rows with 256 bins: the epilogue sweep's dynamic shared memory
    # is exactly 48 KB, plus its static barriers
    ((256, 256), "power", "f32", "poisson"),
    ((64, 64, 64), "power", "f32", "gauss"),
    ((4096,), "power", "f32", "gauss"),
    ((1024, 1024), "power", "f32", "gauss"),
    ((2048, 16), "power", "f32", "poisson"),
    ((16, 2048), "power", "f32", "poisson"),
    ((64, 32), "matern_model", "f64", "poisson"),
    ((512, 512), "matern_model", "f32", "poisson"),
    ((32, 32, 32), "matern_model", "f32", "gauss"),
])
def test_metric_apply(shape, kind, dtype, lik):
    plan, om, M, xi_p, w = _setup(shape, kind, dtype, lik)
    B = 3
    v = rounded(np.random.default_rng(5).standard_normal((B, om.latent_size)), dtype)
    out = host(M.apply(to_dev(plan, v)), om.latent_size)
    tol = 1e-12 if dtype == "f64" else 1e-5
    for b in range(B):
        assert blocks_rel(out[b], ometric(om, xi_p, w, v[b]), om.n_field) <= tol


def test_metric_masked_gaussian_3d():
    shape = (16, 32, 16)
    n = int(np.prod(shape))
    mask = synth.mask_fraction(synth.SEED_MASK, n, 0.1)
    plan, om, M, xi_p, w = _setup(shape, "power", "f32", "gauss", mask=mask, sigma=0.05)
    v = rounded(np.random.default_rng(6).standard_normal((2, om.latent_size)), "f32")
    out = host(M.apply(to_dev(plan, v)), om.latent_size)
    for b in range(2):
        assert blocks_rel(out[b], ometric(om, xi_p, w, v[b]), om.n_field) <= 1e-5


def test_metric_full_size_3d_256_sampled():
    """3-D 256^3 (the largest workload) at batch 1: the whole product against the
    oracle's (FFT-based, a few seconds)."""
    shape = (256, 256, 256)
    n = int(np.prod(shape))
    mask = synth.mask_fraction(synth.SEED_MASK, n, 0.1)
    plan, om, M, xi_p, w = _setup(shape, "power", "f32", "gauss", mask=mask, sigma=0.05, max_batch=1)
    v = rounded(synth.normal(synth.SEED_TANGENT, om.latent_size), "f32")
    out = host(M.apply(to_dev(plan, v[None])), om.latent_size)[0]
    ref = ometric(om, xi_p, w, v)
    assert blocks_rel(out, ref, om.n_field) <= 1e-5


@pytest.mark.parametrize("shape,kind,dtype,lik", [
    ((256,), "matern", "f64", "gauss"),
    ((64, 32), "power", "f64", "poisson"),
    ((512, 512), "power", "f32", "poisson"),
    ((8, 16, 32), "power", "f32", "gauss"),
])
def test_mgvi_rhs(shape, kind, dtype, lik):
    plan, om, M, xi_p, w = _setup(shape, kind, dtype, lik)
    g = np.random.default_rng(8)
    xp = rounded(g.standard_normal((2, om.latent_size)), dtype)
    eta = rounded(g.standard_normal((2, om.n_field)), dtype)
    b = host(M.mgvi_rhs(to_dev(plan, xp), torch.tensor(eta, dtype=plan.dtype, device=DEV)), om.latent_size)
    tol = 1e-12 if dtype == "f64" else 1e-5
    for i in range(2):
        assert blocks_rel(b[i], orhs(om, xi_p, w, xp[i], eta[i]), om.n_field) <= tol


def test_cg_config1_per_iteration():
    """1-D N=256, FP64, fixed spectrum, Gaussian sigma 0.1 at p = xi_true: the
    50-iteration solve.

    CG iterates are chaotic under rounding: perturbing b by one ulp changes the
    oracle's own iterate at k = 20 by ~3e-4.  So (a) while the oracle's
    one-ulp sensitivity is below 1e-13 (k <= 10 here) the GPU iterate must
    match to 1e-12 * max(1, kappa_hat); (b) at every k the GPU iterate must be
    as good in the energy norm ||x_k - x*||_M as the oracle's (CG optimality)
    up to the spread the oracle shows under one-ulp perturbations of b."""
    from oracle.metric import dense_metric
    plan, om, M, xi_p, w = _setup((256,), "matern", "f64", "gauss", seed=synth.SEED_TRUTH)
    b = synth.normal(synth.SEED_RHS, 256)
    kappa = lanczos_kappa(om, xi_p, w, b, 50)
    Md = dense_metric(om, xi_p, w)
    xs = np.linalg.solve(Md, b)
    enorm = lambda x: np.sqrt((x - xs) @ Md @ (x - xs) / (xs @ Md @ xs))
    runs = []
    for t in range(3):
        bp = b if t == 0 else b * (1 + 1e-16 * np.random.default_rng(t).standard_normal(256))
        hist = {}
        ocg(lambda p: ometric(om, xi_p, w, p), bp, rtol=0.0, maxiter=50,
            callback=lambda k, x: hist.__setitem__(k, x.copy()))
        runs.append(hist)
    for k in [1, 2, 5, 10, 15, 20, 25, 35, 50]:
        x, its, rel, st = M.cg(to_dev(plan, b), rtol=0.0, maxiter=k)
        assert its[0] == k
        xg = host(x, 256)[0]
        sens = max(rel_l2(runs[t][k], runs[0][k]) for t in (1, 2))
        if sens < 1e-13:
            assert rel_l2(xg, runs[0][k]) <= 1e-12 * max(1.0, kappa), (k, rel_l2(xg, runs[0][k]))
        e_or = [enorm(runs[t][k]) for t in range(3)]
        spread = max(e_or) - min(e_or)
        assert enorm(xg) <= max(e_or) + 10 * spread + 1e-12, (k, enorm(xg), e_or)


def test_cg_batched_fp64_2d_converges():
    plan, om, M, xi_p, w = _setup((32, 32), "power", "f64", "poisson", max_batch=3)
    g = np.random.default_rng(9)
    b = g.standard_normal((3, om.latent_size))
    x, its, rel, st = M.cg(to_dev(plan, b), rtol=1e-10, maxiter=2000)
    assert st == 0
    xs = host(x, om.latent_size)
    for i in range(3):
        assert rel[i] <= 1e-10
        true = rel_l2(ometric(om, xi_p, w, xs[i]), b[i])
        assert true <= 1e-9
        xr, _, _ = ocg(lambda p: ometric(om, xi_p, w, p), b[i], rtol=1e-12, maxiter=5000)
        assert rel_l2(xs[i], xr) <= 1e-7


def test_pcg_fp32_512_true_residual():
    """2-D 512^2 Poisson, FP32 vectors with FP64 reductions, the harmonic
    preconditioner: a batched solve to recursive ||r|| / ||b|| <= 1e-5.

    The true residual of an FP32 solution is bounded by
        ||b - M x|| <= ||b - M32 x|| + ||(M32 - M) x||,
    the residual the FP32 solver drives down plus the FP32 operator's error on
    x.  The first term is the recursive residual plus the drift of k FP32
    updates of x (a random walk of one-ulp roundings, sqrt(k) times the
    one-ulp floor ||M d|| for d = x * 2^-24 * (+-1)); the second is measured
    directly: the GPU's FP32 product M32 x against the oracle's FP64 M x."""
    plan, om, M, xi_p, w = _setup((512, 512), "power", "f32", "poisson", max_batch=2)
    M.set_precond("harmonic")
    b = rounded(np.random.default_rng(10).standard_normal((2, om.latent_size)), "f32")
    x, its, rel, st = M.cg(to_dev(plan, b), rtol=1e-5, maxiter=500)
    assert st == 0, (its, rel)
    assert max(its) < 200 and max(rel) <= 1e-5
    xs = host(x, om.latent_size)
    mx32 = host(M.apply(x), om.latent_size)
    g = np.random.default_rng(13)
    for i in range(2):
        nb = np.linalg.norm(b[i])
        mx = ometric(om, xi_p, w, xs[i])
        true = np.linalg.norm(mx - b[i]) / nb
        op = np.linalg.norm(mx32[i] - mx) / nb
        d = xs[i] * 2.0 ** -24 * g.choice([-1.0, 1.0], size=xs[i].shape)
        floor = np.linalg.norm(ometric(om, xi_p, w, d)) / nb
        bound = rel[i] + op + 2 * np.sqrt(its[i]) * floor
        assert true <= 1.5 * bound, (i, true, rel[i], op, floor, its[i])


@pytest.mark.parametrize("shape,kind,lik", [((256,), "matern", "gauss"), ((32, 32), "power", "poisson"),
                                            ((16, 16, 16), "power", "gauss")])
def test_pcg_fp64_matches_plain_solution(shape, kind, lik):
    """The preconditioner changes the iterates, not the solution: FP64 PCG to
    1e-11 agrees with the oracle's plain CG solution."""
    plan, om, M, xi_p, w = _setup(shape, kind, "f64", lik, max_batch=2)
    M.set_precond("harmonic")
    b = np.random.default_rng(12).standard_normal((2, om.latent_size))
    x, its, rel, st = M.cg(to_dev(plan, b), rtol=1e-11, maxiter=3000)
    assert st == 0, (its, rel)
    xs = host(x, om.latent_size)
    for i in range(2):
        assert rel_l2(ometric(om, xi_p, w, xs[i]), b[i]) <= 1e-10
        xr, _, _ = ocg(lambda p: ometric(om, xi_p, w, p), b[i], rtol=1e-13, maxiter=20000)
        assert rel_l2(xs[i], xr) <= 1e-8


def test_cg_fp32_power_model_iterates():
    """FP32 plain CG on the 2-D power-model Poisson metric, where the CG
    kernels take over the metric product's hyper-parameter block (q_h from the
    bin sums, p.q's hyper part as p_h.p_h + dA.g, the next dA in the p-update):
    the iterates match the oracle's FP64 CG iterates, field and hyper blocks
    separately.  This metric is so ill-conditioned (relres 30-60 after one
    iteration) that CG amplifies rounding fast: iterates 1 and 2 must match to
    the FP32 product tolerance 1e-5 (measured <= 5e-7); iterate 4 must lie
    within ten times the spread of oracle runs whose products carry a seeded
    relative error of 1e-6 (the FP32 product's size), as CG's chaos allows no
    fixed bound (measured: GPU 2e-6 / 8e-5, spread 1e-4 / 2e-4)."""
    plan, om, M, xi_p, w = _setup((64, 64), "power", "f32", "poisson", max_batch=2)
    b = rounded(np.random.default_rng(14).standard_normal((2, om.latent_size)), "f32")
    mv = lambda p: ometric(om, xi_p, w, p)
    for k in (1, 2, 4):
        x, its, rel, st = M.cg(to_dev(plan, b), rtol=0.0, maxiter=k)
        assert its == [k, k] and st == 0
        xs = host(x, om.latent_size)
        for i in range(2):
            xr, _, rr = ocg(mv, b[i], rtol=0.0, maxiter=k)
            e = blocks_rel(xs[i], xr, om.n_field)
            if k <= 2:
                assert e <= 1e-5, (k, i, e)
                assert abs(rel[i] - rr) <= 1e-5 * rr, (k, i, rel[i], rr)
                continue
            g = np.random.default_rng(100 + i)

            def noisy(p):
                y = mv(p)
                return y + 1e-6 * np.linalg.norm(y) / np.sqrt(y.size) * g.standard_normal(y.shape)

            spread = max(blocks_rel(ocg(noisy, b[i], rtol=0.0, maxiter=k)[0], xr, om.n_field) for _ in range(3))
            assert e <= 10 * spread, (k, i, e, spread)


def test_cg_fixed_iterations_and_notconv():
    plan, om, M, xi_p, w = _setup((64, 64), "power", "f32", "poisson", max_batch=2)
    b = rounded(np.random.default_rng(11).standard_normal((2, om.latent_size)), "f32")
    x, its, rel, st = M.cg(to_dev(plan, b), rtol=0.0, maxiter=7)
    assert its == [7, 7] and st == 0
    x, its, rel, st = M.cg(to_dev(plan, b), rtol=1e-12, maxiter=3)
    assert st == 4  # NRE_ENOTCONV


@pytest.mark.parametrize("shape,lik", [((128, 128), "poisson"), ((32, 32, 32), "gauss"), ((4096,), "poisson")])
def test_products_and_cg_bitwise_repeatable(shape, lik):
    """Every reduction of the FP32 path adds in a fixed order (warp-private
    bin histograms folded in warp, then CTA order; inner products per block in
    a fixed tree): the same inputs give bitwise the same metric products and
    CG iterates, on one metric object and on a second one built alike."""
    import paper_2402_16683_gb300 as nre
    outs, xs = [], []
    for rep in range(2):
        plan, om, M, xi_p, w = _setup(shape, "power", "f32", lik, max_batch=6)
        v = to_dev(plan, rounded(np.random.default_rng(15).standard_normal((6, om.latent_size)), "f32"))
        o1 = M.apply(v).clone()
        o2 = M.apply(v).clone()
        assert torch.equal(o1, o2)
        x, its, rel, st = M.cg(v, rtol=0.0, maxiter=40)
        x1 = x.clone()
        x, its2, rel2, st = M.cg(v, rtol=0.0, maxiter=40)
        assert torch.equal(x1, x) and rel == rel2
        outs.append(o1)
        xs.append(x1)
    assert torch.equal(outs[0], outs[1]) and torch.equal(xs[0], xs[1])


def test_cg_matern_model_fp64_converges_and_fp32_iterates():
    """CG on the metric of the parametric Matern amplitude: FP64 to 1e-10 (true
    residual from the oracle, distance to the oracle's solution), FP32 plain CG
    (the three hyper-parameters inside the CG kernels) at iterates 1 and 2 to
    the product tolerance."""
    plan, om, M, xi_p, w = _setup((32, 32), "matern_model", "f64", "poisson", max_batch=2)
    b = np.random.default_rng(16).standard_normal((2, om.latent_size))
    x, its, rel, st = M.cg(to_dev(plan, b), rtol=1e-10, maxiter=3000)
    assert st == 0
    xs = host(x, om.latent_size)
    for i in range(2):
        assert rel_l2(ometric(om, xi_p, w, xs[i]), b[i]) <= 1e-9
        xr, _, _ = ocg(lambda p: ometric(om, xi_p, w, p), b[i], rtol=1e-12, maxiter=5000)
        assert rel_l2(xs[i], xr) <= 1e-7
    plan, om, M, xi_p, w = _setup((64, 64), "matern_model", "f32", "poisson", max_batch=2)
    b = rounded(np.random.default_rng(17).standard_normal((2, om.latent_size)), "f32")
    for k in (1, 2):
        x, its, rel, st = M.cg(to_dev(plan, b), rtol=0.0, maxiter=k)
        xs = host(x, om.latent_size)
        for i in range(2):
            xr, _, _ = ocg(lambda p: ometric(om, xi_p, w, p), b[i], rtol=0.0, maxiter=k)
            assert blocks_rel(xs[i], xr, om.n_field) <= 1e-5, (k, i)


@pytest.mark.parametrize("shape,kind,lik", [((64, 64), "power", "poisson"), ((512, 512), "power", "poisson"),
                                            ((32, 32, 32), "power", "gauss"), ((128, 128), "matern_model", "poisson")])
def test_cg_refined_true_residual(shape, kind, lik):
    """Residual correction: FP32 inner CG, FP64 residuals.  The oracle's FP64
    true residual ||b - M x|| / ||b|| of the result is <= 1e-5 for every
    system and equals the one the library reports; a plain FP32 solve to the
    same recursive tolerance is printed beside it for comparison."""
    import paper_2402_16683_gb300 as nre
    plan, om, M32, xi_p, w = _setup(shape, kind, "f32", lik, max_batch=2)
    plan64, _ = cf_pair(shape, kind, "f64")
    L, _ = _lik(nre, lik, om)
    M64 = nre.Metric(plan64, L, to_dev(plan64, xi_p)[0], max_batch=2)
    b = np.random.default_rng(18).standard_normal((2, om.latent_size))
    x, its, rel, outer, st = M32.cg_refined(M64, to_dev(plan64, b), rtol=1e-5, max_outer=6, inner_rtol=1e-3,
                                            inner_maxiter=3000)
    assert st == 0 and 1 <= outer <= 6, (st, outer, rel)
    xs = host(x, om.latent_size)
    xp, _, relp, _ = M32.cg(to_dev(plan, rounded(b, "f32")), rtol=1e-5, maxiter=3000)
    xps = host(xp, om.latent_size)
    for i in range(2):
        true = rel_l2(ometric(om, xi_p, w, xs[i]), b[i])
        plain = rel_l2(ometric(om, xi_p, w, xps[i]), b[i])
        print(f"{shape} {kind} {lik} system {i}: passes {outer}, inner iterations {its[i]}, true relres {true:.2e} "
              f"(reported {rel[i]:.2e}); plain FP32 CG to recursive 1e-5: true {plain:.2e}")
        assert true <= 1e-5, (i, true)
        assert abs(true - rel[i]) <= 1e-3 * true + 1e-12, (i, true, rel[i])
