"""Hartley transform on a regular grid (oracle; test infrastructure only).

Sec. "Gaussian Processes" writes a correlated-field draw as s = FT o sqrt(P) o xi
with FT a fast Fourier transform on the regular grid.  Reading: FT is the real,
unnormalised, multi-dimensional discrete Hartley transform

    H[z]_k = sum_x z_x cas(2 pi sum_d k_d x_d / N_d),   cas = cos + sin,

over integer indices.  It is symmetric (H^T = H) and H H = N I.  With the
forward DFT X = sum_x z_x exp(-2 pi i k.x/N) one has H[z] = Re X - Im X, so the
library FFT (numpy.fft.fftn) serves as the single step here.
"""
import numpy as np


def dht(z):
    """Unnormalised multi-dimensional DHT over all axes of ``z`` (float64)."""
    x = np.fft.fftn(np.asarray(z, dtype=np.float64))
    return x.real - x.imag
