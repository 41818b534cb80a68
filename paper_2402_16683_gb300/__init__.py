"""GB300 (sm_103a) library for the NIFTy.re metric-vector-product / CG-sampling
hot path (arXiv:2402.16683): correlated-field and ICR models with hand-written
JVP/VJP kernels, the metric M_p = J^T N^-1 J + 1, MGVI right-hand sides and
batched conjugate gradients, behind the C ABI of include/nre.h.
"""
from ._lib import NREError, load as load_library  # noqa: F401
from .api import ICR, KL, CorrelatedField, Likelihood, Metric, Server, bin_map, device_bytes  # noqa: F401
