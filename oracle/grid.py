"""Harmonic geometry of a regular periodic grid (oracle; test infrastructure only).

Sec. "Gaussian Processes": the correlated field lives on a regular Cartesian
grid whose harmonic domain is reached by an FFT; the example grid has unit
total volume (``distances = 1/d``).  Readings used here:

* axis d has N_d pixels of spacing dx_d; the harmonic index j in [0, N_d) is
  folded to m = j for j <= N_d/2, else j - N_d (the Nyquist index is +N_d/2);
* k_d = m_d / (N_d dx_d) and |k| = sqrt(sum_d k_d^2);
* the power spectrum is binned on l = ln|k| into ``n_bins`` equal-width bins
  between the smallest and the largest non-zero |k|; a pixel with l falls into
  bin min(n_bins-1, floor((l - l_min)/dl)), and the zero mode k = 0 belongs to
  no bin (it carries the offset).  If every non-zero |k| is equal, dl := 1 and
  all such pixels fall into bin 0.
"""
import numpy as np


def folded_index(n):
    """Folded harmonic index m for j = 0..n-1."""
    j = np.arange(n)
    return np.where(j <= n // 2, j, j - n)


def k_norm(shape, spacing):
    """|k| for every harmonic pixel, C order, float64."""
    shape = tuple(int(s) for s in shape)
    ks = []
    for d, n in enumerate(shape):
        m = folded_index(n).astype(np.float64)
        k = m / (n * float(spacing[d]))
        sh = [1] * len(shape)
        sh[d] = n
        ks.append(k.reshape(sh))
    k2 = np.zeros(shape)
    for k in ks:
        k2 = k2 + k * k
    return np.sqrt(k2)


class LogBins:
    """The log-|k| binning of the amplitude model.

    Attributes: ``index`` (int64 array of the grid shape, -1 at k = 0),
    ``centres`` l_i, ``counts`` n_b (number of non-zero modes per bin),
    ``l_min``, ``dl``.
    """

    def __init__(self, shape, spacing, n_bins=256):
        kn = k_norm(shape, spacing)
        nz = kn > 0
        if not np.any(nz):
            raise ValueError("grid has no non-zero harmonic mode")
        l = np.zeros_like(kn)
        l[nz] = np.log(kn[nz])
        l_min = float(l[nz].min())
        l_max = float(l[nz].max())
        dl = (l_max - l_min) / n_bins
        if dl == 0.0:
            dl = 1.0
        idx = np.full(kn.shape, -1, dtype=np.int64)
        b = np.floor((l[nz] - l_min) / dl).astype(np.int64)
        idx[nz] = np.minimum(b, n_bins - 1)
        self.index = idx
        self.n_bins = int(n_bins)
        self.l_min = l_min
        self.dl = dl
        self.centres = l_min + (np.arange(n_bins) + 0.5) * dl
        self.counts = np.bincount(idx[nz], minlength=n_bins).astype(np.float64)
