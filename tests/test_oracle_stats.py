"""Pins for the oracle's quality measures and matter statistics.

* Gaussian smoothing: a single Fourier mode is multiplied by
  exp(-|k|^2 r^2 / 2) exactly; the mean is kept; radius 0 is the identity.
* r and D_Euc: r(a, c a) = sign(c), r of two different modes is 0,
  D_Euc(a, a + c) = |c| for a constant c.
* Moments and histogram of ln(1 + delta) against scipy.stats and
  numpy.histogram on explicit edges.
"""
import math

import numpy as np
import pytest

from oracle import stats


def _mode(n, m):
    i = np.arange(n)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return np.cos(2 * math.pi * (m[0] * z + m[1] * y + m[2] * x) / n)


@pytest.mark.parametrize("n,m,radius", [(16, (0, 1, 3), 4.0), (12, (2, 5, 6), 1.5), (8, (4, 4, 4), 0.7)])
def test_smoothing_of_a_single_mode(n, m, radius):
    box = 3.0 * n
    f = _mode(n, m)
    k = 2 * math.pi / box * math.sqrt(sum((mi if mi < (n + 1) // 2 else mi - n) ** 2 for mi in m))
    out = stats.gaussian_smooth(f, box, radius)
    assert np.max(np.abs(out - math.exp(-0.5 * (k * radius) ** 2) * f)) <= 1e-13


def test_smoothing_keeps_the_mean_and_radius_zero_is_identity():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((10, 10, 10)) + 3.0
    s = stats.gaussian_smooth(x, 50.0, 6.0)
    assert abs(s.mean() - x.mean()) <= 1e-13
    assert np.max(np.abs(stats.gaussian_smooth(x, 50.0, 0.0) - x)) <= 1e-13
    assert s.std() < x.std()


def test_correlation_and_distance():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((8, 8, 8))
    assert abs(stats.correlation(a, 3.0 * a) - 1.0) <= 1e-14
    assert abs(stats.correlation(a, -0.5 * a) + 1.0) <= 1e-14
    assert abs(stats.correlation(_mode(8, (1, 0, 0)), _mode(8, (0, 2, 0)))) <= 1e-14
    assert abs(stats.euclidean_distance(a, a + 0.25) - 0.25) <= 1e-14


def test_log_stats_against_scipy_and_numpy():
    sp = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    n = 12
    lo, width, nbins = -3.0, 0.2, 30
    # values of ln(1 + delta) away from the bin edges, plus out-of-range and invalid cells
    j = rng.integers(-3, nbins + 3, size=n ** 3)
    x = lo + (j + 0.5 + 0.3 * rng.uniform(-1, 1, size=n ** 3)) * width
    delta = np.exp(x) - 1.0
    delta[:7] = -1.5                      # 1 + delta <= 0
    delta = delta.reshape(n, n, n)
    counts, below, above, invalid, mean, var, skew, kurt = stats.log_density_stats(delta, lo, width, nbins)
    xv = x[7:]
    edges = lo + width * np.arange(nbins + 1)
    assert np.array_equal(counts, np.histogram(xv, bins=edges)[0])
    assert below == int(np.sum(xv < lo)) and above == int(np.sum(xv >= edges[-1]))
    assert invalid == 7
    assert abs(mean - xv.mean()) <= 1e-13 and abs(var - xv.var()) <= 1e-12
    assert abs(skew - sp.skew(xv)) <= 1e-12
    assert abs(kurt - sp.kurtosis(xv, fisher=True)) <= 1e-12
