"""Pins of the oracle's Hartley transform and harmonic grid (CPU only).

The transform is pinned by the hand-computed length-4 table, a brute-force
O(N^2) evaluation of the cas-of-the-sum definition on tiny grids, the
involution H H = N I and Parseval.
"""
import os

import numpy as np
import pytest

from oracle.dht import dht
from oracle.grid import LogBins, folded_index, k_norm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_dht(z):
    """sum_x z_x cas(2 pi sum_d k_d x_d / N_d), evaluated pixel by pixel."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    for k in np.ndindex(z.shape):
        acc = 0.0
        for x in np.ndindex(z.shape):
            ang = 2.0 * np.pi * sum(k[d] * x[d] / z.shape[d] for d in range(z.ndim))
            acc += z[x] * (np.cos(ang) + np.sin(ang))
        out[k] = acc
    return out


def test_dht_length4_table():
    tab = np.loadtxt(os.path.join(GOLDEN, "dht_n4.txt"))
    for x in range(4):
        e = np.zeros(4)
        e[x] = 1.0
        np.testing.assert_allclose(dht(e), tab[:, x], atol=1e-15)


@pytest.mark.parametrize("shape", [(2,), (4,), (8,), (16,), (3,), (5,), (4, 4), (8, 4),
                                   (2, 6), (4, 4, 4), (2, 4, 8), (3, 2, 5)])
def test_dht_brute_force(shape):
    z = np.random.default_rng(11).standard_normal(shape)
    np.testing.assert_allclose(dht(z), brute_dht(z), rtol=0, atol=1e-12 * np.abs(z).sum())


@pytest.mark.parametrize("shape", [(64,), (16, 8), (8, 4, 16), (256,)])
def test_dht_involution_and_parseval(shape):
    z = np.random.default_rng(12).standard_normal(shape)
    n = z.size
    hz = dht(z)
    np.testing.assert_allclose(dht(hz), n * z, rtol=0, atol=1e-13 * n * np.abs(z).max() * 10)
    assert abs(np.sum(hz * hz) - n * np.sum(z * z)) <= 1e-12 * n * np.sum(z * z)


def test_dht_symmetric_matrix():
    n = 6
    H = np.stack([dht(np.eye(n)[i]) for i in range(n)], axis=1)
    np.testing.assert_allclose(H, H.T, atol=1e-14)


def test_folded_index_and_knorm():
    assert list(folded_index(8)) == [0, 1, 2, 3, 4, -3, -2, -1]
    assert list(folded_index(5)) == [0, 1, 2, -2, -1]
    kn = k_norm((4, 8), (0.25, 0.125))      # unit volume: k = m
    assert kn[0, 0] == 0.0
    assert kn[1, 0] == 1.0 and kn[0, 7] == 1.0
    assert np.isclose(kn[2, 4], np.sqrt(4 + 16))
    kn2 = k_norm((8,), (0.5,))              # L = 4: k = m / 4
    np.testing.assert_allclose(kn2, np.abs(folded_index(8)) / 4.0)


def test_log_bins():
    b = LogBins((32, 32), (1 / 32, 1 / 32), n_bins=16)
    assert b.index[0, 0] == -1
    assert b.counts.sum() == 32 * 32 - 1
    kn = k_norm((32, 32), (1 / 32, 1 / 32))
    order = np.argsort(kn.ravel(), kind="stable")
    bins_sorted = b.index.ravel()[order][1:]
    assert np.all(np.diff(bins_sorted) >= 0)          # monotone in |k|
    assert bins_sorted[0] == 0 and bins_sorted[-1] == 15
    np.testing.assert_allclose(b.centres[1] - b.centres[0], b.dl)
    # smallest |k| (=1) sits in bin 0, largest (=16 sqrt 2) in the last bin
    assert b.index[1, 0] == 0 and b.index[16, 16] == 15


def test_log_bins_degenerate():
    b = LogBins((2,), (0.5,), n_bins=4)     # only |k| = 1 besides the zero mode
    assert list(b.index) == [-1, 0]
    assert b.dl == 1.0
