"""Checks on the seeded input generator (Philox, fields, counts, selection)."""
import math
import os

import numpy as np
import pytest

from paper_0911_1407_gb300 import mocks

KAT = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    for line in open(KAT):
        if not line.strip() or line.startswith("#"):
            continue
        words = [int(x, 16) for x in line.split()]
        ctr, key, out = words[:4], words[4:6], words[6:]
        got = mocks.philox4x32_10(*ctr, *key)
        assert [int(g) for g in got] == out


def test_uniforms_open_interval_and_moments():
    u1, u2 = mocks.uniform_pair(np.arange(200000), 0, 0, 7, 0)
    for u in (u1, u2):
        assert u.min() > 0 and u.max() < 1
        assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    assert abs(np.corrcoef(u1, u2)[0, 1]) < 0.01


def test_white_noise_moments():
    z = mocks.white_noise(64, seed=3)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01


def test_gaussian_field_variance_and_zero_mean():
    n, box, sig = 32, 200.0, 1.0
    A = mocks.amplitude_for_sigma(n, box, sig)
    var = [mocks.gaussian_field(n, box, A, seed=s).var() for s in range(1, 9)]
    assert abs(np.mean(var) - sig ** 2) < 0.1
    assert abs(mocks.gaussian_field(n, box, A, seed=1).mean()) < 1e-12


def test_poisson_counts_moments_and_determinism():
    for lam in (0.3, 4.0, 75.0):
        c = mocks.poisson_counts(np.full(200000, lam), seed=5)
        assert abs(c.mean() - lam) < 5 * math.sqrt(lam / c.size)
        assert abs(c.var() / lam - 1) < 0.03
    lam = np.exp(np.random.default_rng(0).standard_normal(5000) * 2)
    a = mocks.poisson_counts(lam, seed=9)
    b = mocks.poisson_counts(lam, seed=9)
    c = mocks.poisson_counts(lam, seed=10)
    assert a.dtype == np.int32 and np.array_equal(a, b) and not np.array_equal(a, c)
    assert mocks.poisson_counts(np.zeros(10), seed=1).sum() == 0


def test_selection_mask_fraction():
    w = mocks.radial_masked_selection(64, 500.0, seed=1)
    assert w.min() >= 0 and w.max() <= 1
    zero = (w == 0).mean()
    assert 0.12 < zero < 0.28     # 102 of 512 equal-area patches


def test_table_covers_grid_and_workloads():
    for spec in mocks.WORKLOADS.values():
        kf = 2 * math.pi / spec.box
        A = 1.0
        k, P = mocks.pk_table(spec.n, spec.box, A, spec.nbins)
        assert k[0] <= kf and k[-1] >= math.sqrt(3) * math.pi * spec.n / spec.box
        assert np.all(P > 0) and np.all(np.diff(k) > 0)


def test_mock_plain32_shape():
    m = mocks.make_mock(mocks.WORKLOADS["plain32"])
    assert m.N.shape == (32, 32, 32) and m.N.dtype == np.int32 and m.w is None
    assert abs(m.N.mean() - 2.0) < 0.2 and m.mu == -0.5


def test_batch_specs():
    specs = mocks.batch_specs()
    assert len(specs) == 64
    assert sorted({s.n for s in specs}) == [64, 96, 128]
    assert all(0.8 <= s.sigma_G <= 1.8 and 0.2 <= s.nbar <= 2 for s in specs)
    assert len({s.seed for s in specs}) == 64
