"""Pins for the oracle's Lambert W (used by the diagonal-prior closed form)."""
import math
import os

import numpy as np
import pytest

from oracle.lambertw import lambertw, lambertw_from_log

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lambertw_values.txt")


def test_golden_values():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for x, wx in rows:
        assert abs(float(lambertw(float(x))) - float(wx)) <= 1e-15 * max(1.0, float(wx))


def test_defining_identity():
    x = np.logspace(-12, 10, 300)
    w = lambertw(x)
    assert np.all(w >= 0)
    assert np.allclose(w * np.exp(w), x, rtol=1e-14, atol=0)
    big = np.logspace(10, 300, 100)
    wb = lambertw(big)
    assert np.allclose(wb + np.log(wb), np.log(big), rtol=1e-15, atol=0)


def test_log_space_identity_for_huge_arguments():
    lx = np.array([5.0, 50.0, 700.0, 1e4, 1e6])
    w = lambertw_from_log(lx)
    assert np.allclose(w + np.log(w), lx, rtol=1e-15, atol=0)


def test_matches_library():
    special = pytest.importorskip("scipy.special")
    x = np.concatenate([np.logspace(-10, 2, 200), np.logspace(2, 300, 100)])
    ref = special.lambertw(x).real
    assert np.allclose(lambertw(x), ref, rtol=2e-15, atol=0)
