"""ctypes loader of the in-tree CUDA library ``libnre.so`` (C ABI of include/nre.h).

Loading fails loudly: there is no CPU fallback.  Build the library with
``python -m paper_2402_16683_gb300.build`` (``__graft_entry__.build()``).
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnre.so")

NRE_OK, NRE_EINVAL, NRE_ENOMEM, NRE_ECUDA, NRE_ENOTCONV, NRE_ETIMEDOUT, NRE_EBUSY, NRE_EAGAIN = range(8)
NRE_F32, NRE_F64 = 0, 1
NRE_AMP_ARRAY, NRE_AMP_MATERN_FIXED, NRE_AMP_POWER_MODEL, NRE_AMP_MATERN_MODEL = 0, 1, 2, 3
NRE_LIK_GAUSS, NRE_LIK_POISSON = 0, 1
NRE_RESP_EXP, NRE_RESP_IDENTITY = 0, 1
NRE_MODEL_CF, NRE_MODEL_ICR = 0, 1
NRE_PRECOND_NONE, NRE_PRECOND_HARMONIC = 0, 1

STATUS_NAMES = {0: "NRE_OK", 1: "NRE_EINVAL", 2: "NRE_ENOMEM", 3: "NRE_ECUDA", 4: "NRE_ENOTCONV",
                5: "NRE_ETIMEDOUT", 6: "NRE_EBUSY", 7: "NRE_EAGAIN"}


class NREError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class CFAmpParams(C.Structure):
    _fields_ = [("kind", C.c_int), ("amp_array", C.POINTER(C.c_double)),
                ("k0", C.c_double), ("gamma", C.c_double), ("variance", C.c_double),
                ("zero_mode", C.c_double),
                ("fluct_mean", C.c_double), ("fluct_std", C.c_double),
                ("slope_mean", C.c_double), ("slope_std", C.c_double),
                ("flex_mean", C.c_double), ("flex_std", C.c_double),
                ("asp_mean", C.c_double), ("asp_std", C.c_double),
                ("offset_mean", C.c_double), ("offset_std", C.c_double),
                ("n_bins", C.c_int),
                ("scale_mean", C.c_double), ("scale_std", C.c_double),
                ("cutoff_mean", C.c_double), ("cutoff_std", C.c_double),
                ("lls_mean", C.c_double), ("lls_std", C.c_double)]


class ICRChartParams(C.Structure):
    _fields_ = [("n0", C.c_int), ("r_min", C.c_double), ("r_max", C.c_double), ("ndim", C.c_int)]


class ICRKernelParams(C.Structure):
    _fields_ = [("rho", C.c_double), ("var", C.c_double)]


class ServeCfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_slots", C.c_int), ("dtype", C.c_int),
                ("chunk_iters", C.c_int), ("use_graphs", C.c_int), ("prep_threads", C.c_int)]


class ServeReq(C.Structure):
    _fields_ = [("ndim", C.c_int), ("shape", C.c_int64 * 3), ("amp", CFAmpParams),
                ("lik_kind", C.c_int), ("response", C.c_int), ("sigma_or_scale", C.c_double),
                ("precond", C.c_int),
                ("n_samples", C.c_int), ("rtol", C.c_double), ("maxiter", C.c_int),
                ("xi_p", C.c_void_p), ("b", C.c_void_p), ("eta", C.c_void_p), ("x_out", C.c_void_p),
                ("refine", C.c_int), ("x64_out", C.c_void_p)]


class ServeResult(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int * 64), ("relres", C.c_double * 64),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("device_bytes", C.c_uint64), ("error", C.c_char * 192)]


class ServeStats(C.Structure):
    _fields_ = [("budget", C.c_uint64), ("reserved", C.c_uint64), ("peak_reserved", C.c_uint64),
                ("active", C.c_int), ("queued", C.c_int), ("idle_objects", C.c_int),
                ("completed", C.c_uint64), ("reused", C.c_uint64), ("created", C.c_uint64),
                ("evicted", C.c_uint64), ("graph_replays", C.c_uint64), ("chunks", C.c_uint64)]


_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)

# name -> (argtypes); every function returns int status except nre_last_error
SIGNATURES = {
    "nre_version": [],
    "cf_create": [C.POINTER(_P), C.c_int, _I64P, C.POINTER(C.c_double), C.POINTER(CFAmpParams), C.c_int],
    "cf_destroy": [_P],
    "cf_latent_layout": [_P, _I64P, _I64P, _I64P, _I64P],
    "cf_latent_size": [_P, _I64P],
    "cf_forward": [_P, _P, _P, C.c_int, _P],
    "cf_jvp": [_P, _P, _P, _P, C.c_int, _P],
    "cf_vjp": [_P, _P, _P, _P, C.c_int, _P],
    "cf_forward_noalloc": [_P, _P, _P, C.c_int, _P],
    "cf_bin_map": [C.c_int, _I64P, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int32)],
    "icr_create": [C.POINTER(_P), C.POINTER(ICRChartParams), C.POINTER(ICRKernelParams), C.c_int, C.c_int],
    "icr_destroy": [_P],
    "icr_latent_layout": [_P, _I64P, _I64P, _I64P],
    "icr_forward": [_P, _P, _P, C.c_int, _P],
    "icr_jvp": [_P, _P, _P, _P, C.c_int, _P],
    "icr_vjp": [_P, _P, _P, _P, C.c_int, _P],
    "lik_create": [C.POINTER(_P), C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int64, C.c_double],
    "lik_destroy": [_P],
    "metric_create": [C.POINTER(_P), C.c_int, _P, _P, _P, C.c_int, _P],
    "metric_destroy": [_P],
    "metric_apply": [_P, _P, _P, C.c_int, _P],
    "mgvi_rhs": [_P, _P, _P, _P, C.c_int, _P],
    "cg_solve": [_P, _P, _P, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int),
                 C.POINTER(C.c_double), _P],
    "metric_set_precond": [_P, C.c_int, _P],
    "geovi_update": [_P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int),
                     C.POINTER(C.c_double), _P],
    "kl_create": [C.POINTER(_P), _P, _P, C.POINTER(C.c_double), C.c_int64, _P, C.c_int, _P],
    "kl_destroy": [_P],
    "kl_set_position": [_P, _P, C.POINTER(C.c_double), _P],
    "kl_energy_gradient": [_P, C.POINTER(C.c_double), _P, _P],
    "kl_energy_at": [_P, _P, C.POINTER(C.c_double), _P],
    "kl_metric": [_P, C.POINTER(_P)],
    "kl_position": [_P, _P, _P],
    "kl_newton_step": [_P, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                       C.POINTER(C.c_int), _P],
    "kl_minimize": [_P, C.c_double, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), _P],
    "cg_solve_refined": [_P, _P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int,
                         C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int), _P],
    "nre_device_bytes": [_I64P],
    "nre_wait_timeouts": [C.POINTER(C.c_uint), C.c_int],
    "nre_wait_selftest": [C.c_uint, _P],
    "serve_create": [C.POINTER(_P), C.POINTER(ServeCfg)],
    "serve_submit": [_P, C.POINTER(ServeReq), C.POINTER(C.c_uint64)],
    "serve_poll": [_P, C.c_uint64, C.POINTER(ServeResult), C.c_int],
    "serve_footprint": [C.POINTER(ServeReq), C.c_int, C.POINTER(C.c_uint64)],
    "serve_stats": [_P, C.POINTER(ServeStats)],
    "serve_destroy": [_P],
    "nre_prof_enable": [C.c_int],
    "nre_prof_report": [C.c_char_p, C.c_size_t],
}

_lib = None


def load():
    """Load libnre.so (once) and declare its signatures; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2402_16683_gb300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.nre_last_error.argtypes = []
    lib.nre_last_error.restype = C.c_char_p
    lib.nre_launch_count.argtypes = []
    lib.nre_launch_count.restype = C.c_ulonglong
    _lib = lib
    return lib


def check(status):
    if status != NRE_OK:
        raise NREError(status, load().nre_last_error().decode())
    return status
