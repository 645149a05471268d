"""GPU quality measures and matter statistics against the oracle.

Bars: r and D_Euc to 1e-12 relative (FP64 sums in different orders);
smoothing to 1e-12 of the field's maximum (float-float transforms for
four-step lengths, FP64 Stockham otherwise); histogram counts bit-exact (the
test's values of ln(1 + delta) lie at least 0.2 bin widths from every edge,
so the two logarithm implementations take the same bin); moments to 1e-12.
"""
import math

import numpy as np
import pytest
import torch

from oracle import stats
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


@pytest.mark.parametrize("n", [32, 48, 128])
def test_compare(plc, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n))
    b = 0.6 * a + 0.8 * rng.standard_normal((n, n, n))
    c = plc.Context(n, 5.0 * n, "fp64")
    r, d = c.compare(dev(a, torch.float64), dev(b, torch.float64))
    assert abs(r - stats.correlation(a, b)) <= 1e-12
    assert abs(d - stats.euclidean_distance(a, b)) <= 1e-12 * d


@pytest.mark.parametrize("n,precision", [(32, "mixed"), (48, "fp64"), (64, "mixed"), (96, "fp64"),
                                         (256, "mixed")])
def test_smooth(plc, n, precision):
    rng = np.random.default_rng(100 + n)
    x = np.exp(rng.standard_normal((n, n, n))) - 1.0
    box = 500.0 * n / 256
    c = plc.Context(n, box, precision)
    for radius in (5.0, 10.0):
        ref = stats.gaussian_smooth(x, box, radius)
        y = host(c.smooth(dev(x, torch.float64), radius))
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [24, 128])
def test_log_stats(plc, n):
    rng = np.random.default_rng(7 + n)
    lo, width, nbins = -4.0, 0.2, 40
    j = rng.integers(-4, nbins + 4, size=n ** 3)
    xv = lo + (j + 0.5 + 0.3 * rng.uniform(-1, 1, size=n ** 3)) * width
    delta = np.exp(xv) - 1.0
    delta[::97] = -1.25                                # 1 + delta <= 0
    delta = delta.reshape(n, n, n)
    counts, below, above, invalid, mean, var, skew, kurt = stats.log_density_stats(delta, lo, width, nbins)
    c = plc.Context(n, 5.0 * n, "fp64")
    g_counts, g_out, g_mom = c.log_stats(dev(delta, torch.float64), lo, width, nbins)
    assert np.array_equal(g_counts, counts)
    assert g_out == (below, above, invalid)
    for a, b in zip(g_mom, (mean, var, skew, kurt)):
        assert abs(a - b) <= 1e-12 * max(abs(b), 1.0)


def test_reconstruction_quality_on_the_production_mock(plc):
    """r and D_Euc of the MAP against the true field, through the library and
    through the oracle, on the same arrays."""
    m = mocks.make_mock(mocks.WORKLOADS["selection128"])
    c = plc.Context(m.n, m.box, "mixed")
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    res = c.newton_krylov_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar)
    d_map = torch.expm1(res.s)
    d_true = dev(np.expm1(m.s_true), torch.float64)
    r, d = c.compare(d_map, d_true)
    a, b = host(d_map), np.expm1(m.s_true)
    assert abs(r - stats.correlation(a, b)) <= 1e-12
    assert abs(d - stats.euclidean_distance(a, b)) <= 1e-12 * d
    assert 0.0 < r < 1.0


@pytest.mark.parametrize("n,nbins", [(4, 4096), (4, 61), (8, 4096)])
def test_log_stats_many_bins_on_small_grids(plc, n, nbins):
    """More bins than cells: the device counts have their own 4099-entry
    buffer, so any nbins up to 4096 is valid on any grid."""
    rng = np.random.default_rng(nbins + n)
    lo, width = -3.0, 6.0 / nbins
    j = rng.integers(-2, nbins + 2, size=n ** 3)
    xv = lo + (j + 0.5 + 0.3 * rng.uniform(-1, 1, size=n ** 3)) * width
    delta = (np.exp(xv) - 1.0).reshape(n, n, n)
    delta[0, 0, 0] = -2.0                              # one invalid cell
    counts, below, above, invalid, mean, var, skew, kurt = stats.log_density_stats(delta, lo, width, nbins)
    c = plc.Context(n, 5.0 * n, "fp64")
    g_counts, g_out, g_mom = c.log_stats(dev(delta, torch.float64), lo, width, nbins)
    assert np.array_equal(g_counts, counts)
    assert g_out == (below, above, invalid)
    for a, b in zip(g_mom, (mean, var, skew, kurt)):
        assert abs(a - b) <= 1e-12 * max(abs(b), 1.0)


def test_log_stats_rejects_too_many_bins(plc):
    """nbins beyond 4096 is refused on the host before any launch."""
    c = plc.Context(4, 20.0, "fp64")
    delta = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda")
    for nbins in (0, 4097):
        with pytest.raises(plc.PlcError) as e:
            c.log_stats(delta, -1.0, 0.1, nbins)
        assert e.value.status == 1
