"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and describes workload shapes; it holds
none of the method's arithmetic.  Every draw is float64 from numpy's PCG64
(``numpy.random.default_rng(seed)``); a float32 run receives the rounded copy.

Workloads (the paper's benchmark inputs and data file are not available; these
stand in with the structure of its benchmark: a square-grid correlated field,
exponential response, Poisson counts, growing grid sizes):

* ``cf1d``    - 1-D N=256, spacing 1/256, fixed spectrum, Gaussian noise 0.1, FP64.
* ``cf2d``    - 2-D 512x512, spacing 1/512, power-spectrum model, Poisson x10.
* ``icr2d``   - ICR on a log-radial chart refined 8x8 -> 1024x1024 (7 levels).
* ``cf3d``    - 3-D 256^3, spacing 1/256, power-spectrum model, Gaussian noise
                0.05 on a 10% pixel mask.
* ``serve``   - request stream: Poisson arrivals, grid size drawn uniformly from
                {1-D 4096, 2-D 256^2, 2-D 1024^2, 3-D 128^3}, Gaussian / Poisson.
"""
import numpy as np

# Prior (mean, std) pairs of the power-spectrum model used by the 2-D, 3-D and
# serving workloads; offset ~ N(0, 1).
AMP_PRIOR = dict(fluct=(1.0, 0.5), slope=(-3.0, 0.5), flex=(1.0, 0.5),
                 asp=(0.1, 0.05), offset_mean=0.0, offset_std=1.0, n_bins=256)

# Prior (mean, std) pairs of the parametric Matern amplitude (scale and cutoff
# log-normal, the power spectrum's log-log slope normal); offset ~ N(0, 1).
MATERN_PRIOR = dict(scale=(1.0, 0.5), cutoff=(8.0, 2.0), loglogslope=(-4.0, 0.5),
                    offset_mean=0.0, offset_std=1.0, n_bins=256)

# Fixed 1-D spectrum (1 + (k/8)^2)^-1.5, unit variance, zero offset.
FIXED_1D = dict(k0=8.0, gamma=1.5, variance=1.0, zero_mode=0.0)

SEED_TRUTH = 0      # xi_true for the 1-D workload (its expansion point)
SEED_POS = 1        # expansion point p elsewhere
SEED_TANGENT = 2    # tangent v
SEED_MASK = 3       # pixel mask permutation
SEED_RHS = 4        # first seed of right-hand sides / MGVI excitations
SEED_STREAM = 5     # request stream

SERVE_SHAPES = [(4096,), (256, 256), (1024, 1024), (128, 128, 128)]


def rng(seed):
    return np.random.default_rng(int(seed))


def normal(seed, shape):
    """Standard normal float64 array."""
    return rng(seed).standard_normal(shape)


def mask_fraction(seed, n, frac=0.1):
    """Exactly round(frac * n) ones chosen by a seeded permutation (float64 0/1)."""
    k = int(round(frac * n))
    perm = rng(seed).permutation(n)
    m = np.zeros(n)
    m[perm[:k]] = 1.0
    return m


def poisson_arrivals(seed, rate, n):
    """Arrival times (s) of a Poisson process with the given rate."""
    return np.cumsum(rng(seed).exponential(1.0 / rate, size=n))


def request_stream(seed=SEED_STREAM, n=2000, rate=50.0):
    """List of (t_arrival, shape, likelihood kind) for the serving workload."""
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=n))
    shapes = g.integers(0, len(SERVE_SHAPES), size=n)
    kinds = g.integers(0, 2, size=n)
    return [(float(t[i]), SERVE_SHAPES[shapes[i]], "gauss" if kinds[i] == 0 else "poisson")
            for i in range(n)]
