"""Shared helpers of the GPU parity tests: plans and oracle models built from the
same parameters, seeded inputs, and the error measures the tolerances use."""
import numpy as np
import torch

import synth
from oracle import amplitude as oamp
from oracle.cf import CFModel, matern_fixed_amplitude

DEV = "cuda:0"


def tdtype(name):
    return torch.float64 if name == "f64" else torch.float32


def cf_pair(shape, kind, dtype, n_bins=256, prior=None, spacing=None):
    """(GPU plan, oracle model) for the same correlated field."""
    import paper_2402_16683_gb300 as nre
    sp = spacing or tuple(1.0 / s for s in shape)
    if kind == "matern":
        plan = nre.CorrelatedField(shape, sp, amplitude="matern", matern=synth.FIXED_1D, dtype=tdtype(dtype))
        om = CFModel(shape, sp, fixed_amp=matern_fixed_amplitude(shape, sp, **synth.FIXED_1D))
    elif kind == "matern_model":
        pr = dict(synth.MATERN_PRIOR)
        pr["n_bins"] = n_bins
        if prior:
            pr.update(prior)
        plan = nre.CorrelatedField(shape, sp, amplitude="matern_model", prior=pr, dtype=tdtype(dtype))
        om = CFModel(shape, sp, prior=oamp.MaternPrior(**pr))
    else:
        pr = dict(synth.AMP_PRIOR)
        pr["n_bins"] = n_bins
        if prior:
            pr.update(prior)
        plan = nre.CorrelatedField(shape, sp, amplitude="power", prior=pr, dtype=tdtype(dtype))
        om = CFModel(shape, sp, prior=oamp.AmpPrior(**pr))
    return plan, om


def rounded(x, dtype):
    """Inputs as the GPU sees them (float32 runs get the rounded copy), in float64."""
    return np.asarray(x, dtype=np.float32 if dtype == "f32" else np.float64).astype(np.float64)


def to_dev(plan, x):
    """[B, latent] float64 numpy -> padded [B, stride] device tensor of the plan dtype."""
    t = torch.tensor(np.atleast_2d(x), dtype=plan.dtype, device=DEV)
    return plan.pad(t)


def field_to_dev(plan, x):
    return torch.tensor(np.atleast_2d(x), dtype=plan.dtype, device=DEV).contiguous()


def host(t, n=None):
    a = t.detach().double().cpu().numpy()
    return a if n is None else a[:, :n]


def rel_max(got, ref):
    """max |got - ref| / max |ref| (the FP64 and FP32 parity measure)."""
    ref = np.asarray(ref)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(np.asarray(got) - ref)) / (den if den > 0 else 1.0))


def rel_l2(got, ref):
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(np.asarray(got) - ref) / (den if den > 0 else 1.0))


def blocks_rel(got, ref, n_field):
    """rel_max of the field block and of the hyper-parameter block separately."""
    e = [rel_max(got[:n_field], ref[:n_field])]
    if ref.shape[0] > n_field:
        e.append(rel_max(got[n_field:], ref[n_field:]))
    return max(e)


def icr_fp64_tol(n0, n_levels, rho=0.1):
    """FP64 parity tolerance of ICR outputs (rel_max), derived from conditioning.

    Both sides assemble R = K_fc K_cc^-1 and L_D = chol(K_ff - R K_cf) in FP64
    from chart positions and kernel values that may differ in the last bit.  A
    relative perturbation eps64 of the 9x9 neighbourhood matrix moves the solve
    by up to n eps64 kappa(K_cc) (n = 9, a backward-stable solver), and each
    refinement adds its level's error to the output.  Hence
        tol = max(1e-12, 9 eps64 sum_l max_i kappa(K_cc[l, i])).
    Returns (tol, [max kappa per level])."""
    from oracle.icr import ICRChart
    c = ICRChart(n0=n0, n_levels=n_levels, rho=rho)
    kap = []
    for lev in range(n_levels):
        k = 0.0
        for i in range(c.sizes[lev]):
            pc, _ = c.coarse_fine_points(lev, i)
            k = max(k, float(np.linalg.cond(c.kmat(pc, pc))))
        kap.append(k)
    tol = max(1e-12, 9 * np.finfo(np.float64).eps * sum(kap))
    return tol, kap


def icr3_fp64_tol(n0, n_levels, rho):
    """As icr_fp64_tol for the 3-D chart: the neighbourhood matrices are 27 x 27,
    so tol = max(1e-12, 27 eps64 sum_l max_(i,j) kappa(K_cc[l, i, j]))."""
    from oracle.icr3 import ICRChart3D
    c = ICRChart3D(n0=n0, n_levels=n_levels, rho=rho)
    kap = []
    for lev in range(n_levels):
        k = 0.0
        n = c.sizes[lev]
        for i in range(n):
            for j in range(n):
                pc, _ = c.coarse_fine_points(lev, i, j)
                k = max(k, float(np.linalg.cond(c.kmat(pc, pc))))
        kap.append(k)
    return max(1e-12, 27 * np.finfo(np.float64).eps * sum(kap)), kap
