"""Thin Python binding of the C ABI (include/nre.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory and
the current stream.  Latent batches are [batch, stride] CUDA tensors (stride
from the plan; entries beyond ``latent_size`` are padding the library neither
reads nor writes); position-space batches are [batch, N].
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L
from ._lib import check

_DT = {torch.float32: L.NRE_F32, torch.float64: L.NRE_F64}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _need(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def bin_map(shape, spacing, n_bins=256):
    """Host-only: log-|k| bin of every harmonic pixel (-1 at k = 0)."""
    lib = L.load()
    shp = (C.c_int64 * len(shape))(*shape)
    sp = (C.c_double * len(shape))(*spacing)
    out = np.zeros(int(np.prod(shape)), dtype=np.int32)
    check(lib.cf_bin_map(len(shape), shp, sp, n_bins, out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out.reshape(shape)


def _amp_params(amplitude="power", prior=None, matern=None, offset_mean=0.0):
    """nre_cf_amp_params of an amplitude choice (see CorrelatedField); returns
    (params, array kept alive for NRE_AMP_ARRAY or None)."""
    a = L.CFAmpParams()
    arr = None
    if isinstance(amplitude, np.ndarray):
        a.kind = L.NRE_AMP_ARRAY
        arr = np.ascontiguousarray(amplitude, dtype=np.float64).ravel()
        a.amp_array = arr.ctypes.data_as(C.POINTER(C.c_double))
        a.offset_mean = offset_mean
    elif amplitude == "matern":
        m = dict(k0=8.0, gamma=1.5, variance=1.0, zero_mode=0.0)
        m.update(matern or {})
        a.kind = L.NRE_AMP_MATERN_FIXED
        a.k0, a.gamma, a.variance, a.zero_mode = m["k0"], m["gamma"], m["variance"], m["zero_mode"]
        a.offset_mean = offset_mean
    elif amplitude == "power":
        pr = dict(fluct=(1.0, 0.5), slope=(-3.0, 0.5), flex=(1.0, 0.5), asp=(0.1, 0.05),
                  offset_mean=0.0, offset_std=1.0, n_bins=256)
        pr.update(prior or {})
        a.kind = L.NRE_AMP_POWER_MODEL
        a.fluct_mean, a.fluct_std = pr["fluct"]
        a.slope_mean, a.slope_std = pr["slope"]
        a.flex_mean, a.flex_std = pr["flex"]
        a.asp_mean, a.asp_std = pr["asp"]
        a.offset_mean, a.offset_std = pr["offset_mean"], pr["offset_std"]
        a.n_bins = pr["n_bins"]
    elif amplitude == "matern_model":
        pr = dict(scale=(1.0, 0.5), cutoff=(8.0, 2.0), loglogslope=(-4.0, 0.5),
                  offset_mean=0.0, offset_std=1.0, n_bins=256)
        pr.update(prior or {})
        a.kind = L.NRE_AMP_MATERN_MODEL
        a.scale_mean, a.scale_std = pr["scale"]
        a.cutoff_mean, a.cutoff_std = pr["cutoff"]
        a.lls_mean, a.lls_std = pr["loglogslope"]
        a.offset_mean, a.offset_std = pr["offset_mean"], pr["offset_std"]
        a.n_bins = pr["n_bins"]
    else:
        raise ValueError(f"unknown amplitude {amplitude!r}")
    return a, arr


class CorrelatedField:
    """Correlated-field plan (cf_create).

    amplitude: "power" (non-parametric power-spectrum model, ``prior`` dict with
    fluct / slope / flex / asp (mean, std) pairs, offset_mean, offset_std,
    n_bins), "matern_model" (parametric Matern spectrum, ``prior`` dict with
    scale / cutoff / loglogslope (mean, std) pairs, offset_mean, offset_std,
    n_bins), "matern" (fixed spectrum, ``matern`` dict k0 / gamma / variance /
    zero_mode) or a per-pixel numpy array (A_full, harmonic C order).
    """

    def __init__(self, shape, spacing=None, amplitude="power", prior=None, matern=None,
                 offset_mean=0.0, dtype=torch.float32):
        lib = L.load()
        self.shape = tuple(int(s) for s in shape)
        self.spacing = tuple(float(s) for s in (spacing or [1.0 / s for s in self.shape]))
        self.dtype = dtype
        a, self._arr = _amp_params(amplitude, prior, matern, offset_mean)
        h = C.c_void_p()
        shp = (C.c_int64 * len(self.shape))(*self.shape)
        sp = (C.c_double * len(self.shape))(*self.spacing)
        check(lib.cf_create(C.byref(h), len(self.shape), shp, sp, C.byref(a), _DT[dtype]))
        self.handle = h
        nf, nh, ls, st = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        check(lib.cf_latent_layout(h, C.byref(nf), C.byref(nh), C.byref(ls), C.byref(st)))
        self.n_field, self.n_hyper, self.latent_size, self.stride = nf.value, nh.value, ls.value, st.value
        self.n_data = self.n_field
        self.kind = L.NRE_MODEL_CF

    def __del__(self):
        if getattr(self, "handle", None) and L._lib is not None:
            L._lib.cf_destroy(self.handle)
            self.handle = None

    # layout helpers ---------------------------------------------------
    def pad(self, x):
        """[B, latent_size] -> zero-padded [B, stride] (a copy)."""
        out = torch.zeros(x.shape[0], self.stride, dtype=x.dtype, device=x.device)
        out[:, :self.latent_size] = x
        return out

    def unpad(self, x):
        return x[:, :self.latent_size]

    # raw calls ----------------------------------------------------------
    def forward(self, xi):
        B = xi.shape[0]
        _need(xi, self.dtype, (B, self.stride), "xi")
        s = torch.empty(B, self.n_field, dtype=self.dtype, device=xi.device)
        check(L.load().cf_forward(self.handle, _ptr(xi), _ptr(s), B, _stream()))
        return s

    def jvp(self, xi_p, v):
        B = v.shape[0]
        _need(xi_p, self.dtype, (B, self.stride), "xi_p")
        _need(v, self.dtype, (B, self.stride), "v")
        out = torch.empty(B, self.n_field, dtype=self.dtype, device=v.device)
        check(L.load().cf_jvp(self.handle, _ptr(xi_p), _ptr(v), _ptr(out), B, _stream()))
        return out

    def vjp(self, xi_p, ct):
        B = ct.shape[0]
        _need(xi_p, self.dtype, (B, self.stride), "xi_p")
        _need(ct, self.dtype, (B, self.n_field), "ct")
        g = torch.zeros(B, self.stride, dtype=self.dtype, device=ct.device)
        check(L.load().cf_vjp(self.handle, _ptr(xi_p), _ptr(ct), _ptr(g), B, _stream()))
        return g

    def __call__(self, xi):
        """Differentiable cf(xi): backward runs cf_vjp, forward-mode AD runs cf_jvp."""
        return _ModelFn.apply(xi, self)


class ICR:
    """Iterative-charted-refinement plan (icr_create): ndim 2 on the log-radial
    chart, ndim 3 on the spherical log-radial chart."""

    def __init__(self, n0=8, n_levels=7, r_min=0.1, r_max=1.0, rho=0.1, var=1.0, dtype=torch.float32, ndim=2):
        lib = L.load()
        self.dtype = dtype
        self.ndim = ndim
        ch = L.ICRChartParams(n0, r_min, r_max, ndim)
        kp = L.ICRKernelParams(rho, var)
        h = C.c_void_p()
        check(lib.icr_create(C.byref(h), C.byref(ch), C.byref(kp), n_levels, _DT[dtype]))
        self.handle = h
        no, ls, st = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib.icr_latent_layout(h, C.byref(no), C.byref(ls), C.byref(st)))
        self.n_data, self.latent_size, self.stride = no.value, ls.value, st.value
        self.n_field = self.n_data
        self.n_out = self.n_data
        self.kind = L.NRE_MODEL_ICR

    def __del__(self):
        if getattr(self, "handle", None) and L._lib is not None:
            L._lib.icr_destroy(self.handle)
            self.handle = None

    pad = CorrelatedField.pad
    unpad = CorrelatedField.unpad

    def forward(self, xi):
        B = xi.shape[0]
        _need(xi, self.dtype, (B, self.stride), "xi")
        s = torch.empty(B, self.n_out, dtype=self.dtype, device=xi.device)
        check(L.load().icr_forward(self.handle, _ptr(xi), _ptr(s), B, _stream()))
        return s

    def jvp(self, xi_p, v):
        B = v.shape[0]
        _need(v, self.dtype, (B, self.stride), "v")
        out = torch.empty(B, self.n_out, dtype=self.dtype, device=v.device)
        check(L.load().icr_jvp(self.handle, _ptr(v), _ptr(v), _ptr(out), B, _stream()))
        return out

    def vjp(self, xi_p, ct):
        B = ct.shape[0]
        _need(ct, self.dtype, (B, self.n_out), "ct")
        g = torch.zeros(B, self.stride, dtype=self.dtype, device=ct.device)
        check(L.load().icr_vjp(self.handle, _ptr(ct), _ptr(ct), _ptr(g), B, _stream()))
        return g

    def __call__(self, xi):
        return _ModelFn.apply(xi, self)


class _ModelFn(torch.autograd.Function):
    """autograd.Function over a model plan: forward -> *_forward, backward ->
    *_vjp (hand-written adjoint kernels), forward-mode jvp -> *_jvp."""

    @staticmethod
    def forward(xi, plan):
        return plan.forward(xi.contiguous())

    @staticmethod
    def setup_context(ctx, inputs, output):
        xi, plan = inputs
        ctx.plan = plan
        ctx.save_for_backward(xi)
        ctx.save_for_forward(xi)

    @staticmethod
    def backward(ctx, g):
        (xi,) = ctx.saved_tensors
        return ctx.plan.vjp(xi.contiguous(), g.contiguous()), None

    @staticmethod
    def jvp(ctx, xi_t, _plan_t):
        (xi,) = ctx.saved_tensors
        return ctx.plan.jvp(xi.contiguous(), xi_t.contiguous())


class Likelihood:
    """lik_create: "gauss" (sigma, optional 0/1 mask, response "exp"/"identity")
    or "poisson" (rate = scale * exp(cf))."""

    def __init__(self, kind="gauss", sigma=0.1, scale=10.0, mask=None, response="exp", n_data=0):
        lib = L.load()
        k = L.NRE_LIK_GAUSS if kind == "gauss" else L.NRE_LIK_POISSON
        r = L.NRE_RESP_EXP if response == "exp" else L.NRE_RESP_IDENTITY
        val = sigma if kind == "gauss" else scale
        mp = None
        if mask is not None:
            self._mask = np.ascontiguousarray(mask, dtype=np.float64).ravel()
            mp = self._mask.ctypes.data_as(C.POINTER(C.c_double))
            n_data = self._mask.size
        h = C.c_void_p()
        check(lib.lik_create(C.byref(h), k, r, mp, int(n_data), float(val)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and L._lib is not None:
            L._lib.lik_destroy(self.handle)
            self.handle = None


class Metric:
    """metric_create: M_p = J^T N^-1 J + 1 linearised at xi_p ([stride] tensor)."""

    def __init__(self, model, lik, xi_p, max_batch=1):
        lib = L.load()
        self.model = model
        self.lik = lik
        xi_p = xi_p.reshape(-1)
        _need(xi_p, model.dtype, (model.stride,), "xi_p")
        h = C.c_void_p()
        check(lib.metric_create(C.byref(h), model.kind, model.handle, lik.handle, _ptr(xi_p),
                                int(max_batch), _stream()))
        self.handle = h
        self.max_batch = max_batch

    def __del__(self):
        if getattr(self, "handle", None) and L._lib is not None and not getattr(self, "_owner", None):
            L._lib.metric_destroy(self.handle)
            self.handle = None

    def apply(self, v, out=None):
        B = v.shape[0]
        _need(v, self.model.dtype, (B, self.model.stride), "v")
        if out is None:
            out = torch.zeros_like(v)
        check(L.load().metric_apply(self.handle, _ptr(v), _ptr(out), B, _stream()))
        return out

    def mgvi_rhs(self, xi_prime, eta, out=None):
        B = xi_prime.shape[0]
        _need(xi_prime, self.model.dtype, (B, self.model.stride), "xi_prime")
        _need(eta, self.model.dtype, (B, self.model.n_data), "eta")
        if out is None:
            out = torch.zeros_like(xi_prime)
        check(L.load().mgvi_rhs(self.handle, _ptr(xi_prime), _ptr(eta), _ptr(out), B, _stream()))
        return out

    def set_precond(self, kind="harmonic"):
        """Select cg's preconditioner: "harmonic" (correlated field: the exact
        inverse of the metric with w replaced by its mean) or None."""
        k = L.NRE_PRECOND_HARMONIC if kind == "harmonic" else L.NRE_PRECOND_NONE
        check(L.load().metric_set_precond(self.handle, k, _stream()))

    def cg(self, b, rtol=1e-5, maxiter=100, x=None, raise_on_notconv=False):
        """Solve M x = b per row; returns (x, iterations[B], relres[B], status)."""
        B = b.shape[0]
        _need(b, self.model.dtype, (B, self.model.stride), "b")
        if x is None:
            x = torch.zeros_like(b)
        it = (C.c_int * B)()
        rr = (C.c_double * B)()
        st = L.load().cg_solve(self.handle, _ptr(b), _ptr(x), B, float(rtol), int(maxiter), it, rr, _stream())
        if st != L.NRE_OK and (st != L.NRE_ENOTCONV or raise_on_notconv):
            check(st)
        return x, list(it), list(rr), st

    def geovi_update(self, b, delta, xtol=1e-4, maxiter=5, cg_rtol=1e-5, cg_maxiter=500):
        """geoVI nonlinear update of the residuals delta ([B, stride], updated in
        place) for right-hand sides b.  Returns (iterations[B], last mean |step|[B])."""
        B = b.shape[0]
        _need(b, self.model.dtype, (B, self.model.stride), "b")
        _need(delta, self.model.dtype, (B, self.model.stride), "delta")
        it = (C.c_int * B)()
        st = (C.c_double * B)()
        check(L.load().geovi_update(self.handle, _ptr(b), _ptr(delta), B, float(xtol), int(maxiter), float(cg_rtol),
                                    int(cg_maxiter), it, st, _stream()))
        return list(it), list(st)

    def cg_refined(self, hi, b, rtol=1e-5, max_outer=6, inner_rtol=1e-3, inner_maxiter=1000, x=None,
                   raise_on_notconv=False):
        """cg_solve_refined: solve to a true relative residual rtol of the FP64
        metric ``hi`` (same model and expansion point), this metric running the
        inner CG.  b, x: FP64 [B, stride].  Returns (x, inner iterations[B],
        true relres[B], passes, status)."""
        B = b.shape[0]
        _need(b, torch.float64, (B, self.model.stride), "b")
        if x is None:
            x = torch.zeros_like(b)
        it = (C.c_int * B)()
        rr = (C.c_double * B)()
        outer = C.c_int(0)
        st = L.load().cg_solve_refined(self.handle, hi.handle, _ptr(b), _ptr(x), B, float(rtol), int(max_outer),
                                       float(inner_rtol), int(inner_maxiter), it, rr, C.byref(outer), _stream())
        if st != L.NRE_OK and (st != L.NRE_ENOTCONV or raise_on_notconv):
            check(st)
        return x, list(it), list(rr), outer.value, st


class KL:
    """kl_create: the MGVI KL energy of a correlated field for fixed residual
    samples (deltas: [S, stride] tensor), its gradient, the sample-averaged
    metric and Newton-CG steps.  data: host array of the N observations."""

    def __init__(self, model, lik, data, deltas):
        lib = L.load()
        self.model, self.lik = model, lik
        self._data = np.ascontiguousarray(np.asarray(data, dtype=np.float64).ravel())
        S = deltas.shape[0]
        _need(deltas, model.dtype, (S, model.stride), "deltas")
        h = C.c_void_p()
        check(lib.kl_create(C.byref(h), model.handle, lik.handle, self._data.ctypes.data_as(C.POINTER(C.c_double)),
                            self._data.size, _ptr(deltas), S, _stream()))
        self.handle = h
        self.n_samples = S

    def __del__(self):
        if getattr(self, "handle", None) and L._lib is not None:
            L._lib.kl_destroy(self.handle)
            self.handle = None

    def set_position(self, xi_bar):
        _need(xi_bar, self.model.dtype, (self.model.stride,), "xi_bar")
        e = C.c_double()
        check(L.load().kl_set_position(self.handle, _ptr(xi_bar), C.byref(e), _stream()))
        return e.value

    def energy_gradient(self):
        e = C.c_double()
        g = torch.zeros(self.model.stride, dtype=self.model.dtype, device="cuda")
        check(L.load().kl_energy_gradient(self.handle, C.byref(e), _ptr(g), _stream()))
        return e.value, g

    def energy_at(self, xi):
        _need(xi, self.model.dtype, (self.model.stride,), "xi")
        e = C.c_double()
        check(L.load().kl_energy_at(self.handle, _ptr(xi), C.byref(e), _stream()))
        return e.value

    def metric(self):
        """The sample-averaged metric at the position (a Metric owned by this KL)."""
        h = C.c_void_p()
        check(L.load().kl_metric(self.handle, C.byref(h)))
        m = Metric.__new__(Metric)
        m.model, m.lik, m.handle, m.max_batch, m._owner = self.model, self.lik, h, 1, self
        return m

    def position(self):
        x = torch.zeros(self.model.stride, dtype=self.model.dtype, device="cuda")
        check(L.load().kl_position(self.handle, _ptr(x), _stream()))
        return x

    def newton_step(self, cg_rtol=1e-3, cg_maxiter=200):
        """One Newton-CG step: (mean |step|, energy, inner CG iterations)."""
        st, e, it = C.c_double(), C.c_double(), C.c_int()
        check(L.load().kl_newton_step(self.handle, float(cg_rtol), int(cg_maxiter), C.byref(st), C.byref(e),
                                      C.byref(it), _stream()))
        return st.value, e.value, it.value

    def minimize(self, xtol=1e-4, maxiter=35, cg_rtol=1e-3, cg_maxiter=200):
        """Newton-CG until mean |step| <= xtol: (iterations, energy)."""
        it, e = C.c_int(), C.c_double()
        check(L.load().kl_minimize(self.handle, float(xtol), int(maxiter), float(cg_rtol), int(cg_maxiter),
                                   C.byref(it), C.byref(e), _stream()))
        return it.value, e.value


def _host_ptr(a, dtype, n, name):
    """Address of a contiguous host array (numpy or CPU tensor) of n entries."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != dtype or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{name}: need a contiguous CPU tensor of {n} {dtype}")
        return a.data_ptr()
    npdt = np.float32 if dtype == torch.float32 else np.float64
    if not isinstance(a, np.ndarray) or a.dtype != npdt or not a.flags.c_contiguous or a.size != n:
        raise ValueError(f"{name}: need a C-contiguous numpy array of {n} {npdt.__name__}")
    return a.ctypes.data


class Server:
    """Request loop for sampling solves (serve_*): continuous batching of
    correlated-field CG solves of different grids on one device.

    Inputs and outputs are HOST arrays in the server dtype (page-locked CPU
    tensors give asynchronous copies); the server reads / writes them until the
    request is polled, and this object keeps them referenced until then.
    """

    def __init__(self, hbm_budget_bytes=0, max_slots=8, dtype=torch.float32, chunk_iters=8,
                 use_graphs=True, prep_threads=8):
        lib = L.load()
        cfg = L.ServeCfg(int(hbm_budget_bytes), int(max_slots), _DT[dtype], int(chunk_iters),
                         1 if use_graphs else 0, int(prep_threads))
        h = C.c_void_p()
        check(lib.serve_create(C.byref(h), C.byref(cfg)))
        self.handle = h
        self.dtype = dtype
        self._keep = {}

    def _request(self, shape, xi_p, b, x_out, lik, sigma, scale, amplitude, prior, matern, precond,
                 rtol, maxiter, eta, n_samples, check_arrays=True, response="exp", refine=0, x64_out=None):
        r = L.ServeReq()
        r.ndim = len(shape)
        for d, n in enumerate(shape):
            r.shape[d] = int(n)
        r.amp, _ = _amp_params(amplitude, prior, matern)
        r.lik_kind = L.NRE_LIK_GAUSS if lik == "gauss" else L.NRE_LIK_POISSON
        r.response = L.NRE_RESP_IDENTITY if response == "identity" else L.NRE_RESP_EXP
        r.sigma_or_scale = float(sigma if lik == "gauss" else scale)
        r.precond = L.NRE_PRECOND_HARMONIC if precond == "harmonic" else L.NRE_PRECOND_NONE
        r.n_samples = int(n_samples)
        r.rtol = float(rtol)
        r.maxiter = int(maxiter)
        r.refine = int(refine)
        if check_arrays:
            N = int(np.prod(shape))
            nh = {L.NRE_AMP_POWER_MODEL: 4 + 2 * (r.amp.n_bins - 1), L.NRE_AMP_MATERN_MODEL: 3}.get(r.amp.kind, 0)
            lat = N + nh
            r.xi_p = _host_ptr(xi_p, self.dtype, lat, "xi_p")
            r.b = _host_ptr(b, self.dtype, n_samples * lat, "b")
            r.x_out = _host_ptr(x_out, self.dtype, n_samples * lat, "x_out") if x_out is not None else None
            r.eta = _host_ptr(eta, self.dtype, n_samples * N, "eta") if eta is not None else None
            if refine:
                r.x64_out = _host_ptr(x64_out, torch.float64, n_samples * lat, "x64_out")
        return r

    def submit(self, shape, xi_p, b, x_out, lik="gauss", sigma=0.1, scale=10.0, amplitude="power",
               prior=None, matern=None, precond="harmonic", rtol=1e-5, maxiter=1000, eta=None,
               response="exp", refine=0, x64_out=None):
        """Queue one request (b: [n_samples, latent], x_out likewise); returns its id.
        refine > 0: residual correction to a true rtol with up to that many
        passes, the FP64 solutions in x64_out (x_out unused, may be None)."""
        n = int(np.prod(b.shape[:-1])) if len(b.shape) > 1 else 1
        r = self._request(shape, xi_p, b, x_out, lik, sigma, scale, amplitude, prior, matern, precond,
                          rtol, maxiter, eta, n, response=response, refine=refine, x64_out=x64_out)
        rid = C.c_uint64()
        check(L.load().serve_submit(self.handle, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (xi_p, b, x_out, eta, x64_out)
        return rid.value

    def footprint(self, shape, n_samples=8, lik="gauss", amplitude="power", prior=None, matern=None,
                  precond="harmonic", mgvi=False, refine=0):
        """Device bytes a request of this kind is charged."""
        r = self._request(shape, None, None, None, lik, 0.1, 10.0, amplitude, prior, matern, precond, 1e-5,
                          1, None, n_samples, check_arrays=False, refine=refine)
        if mgvi:
            r.eta = 1
        out = C.c_uint64()
        check(L.load().serve_footprint(C.byref(r), _DT[self.dtype], C.byref(out)))
        return out.value

    def poll(self, rid, timeout_ms=-1):
        """Result dict of a finished request, or None while it is pending."""
        res = L.ServeResult()
        st = L.load().serve_poll(self.handle, C.c_uint64(rid), C.byref(res), int(timeout_ms))
        if st == L.NRE_EAGAIN:
            return None
        check(st)
        self._keep.pop(rid, None)
        n = 64
        return dict(status=res.status, iters=list(res.iters[:n]), relres=list(res.relres[:n]),
                    t_submit=res.t_submit, t_start=res.t_start, t_done=res.t_done,
                    device_bytes=res.device_bytes, error=res.error.decode(errors="replace"))

    def stats(self):
        s = L.ServeStats()
        check(L.load().serve_stats(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in L.ServeStats._fields_}

    def close(self):
        if getattr(self, "handle", None) and L._lib is not None:
            L._lib.serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        self.close()


def device_bytes():
    """Device bytes held by the library's own allocations."""
    v = C.c_int64()
    check(L.load().nre_device_bytes(C.byref(v)))
    return v.value
