"""Pins for the oracle's DFT: brute force, Parseval, round trip, library.

The prior operator S^-1 is applied through the DFT (Sec. 2.2: S is a
convolution, diagonal in Fourier space), so the oracle's transform is pinned
first, against the O(N^2) definition on tiny grids including radix-3 sizes.
"""
import numpy as np
import pytest

from oracle import dft


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 3, 3), (6, 6, 6), (2, 3, 4), (5, 2, 3)])
def test_separable_dft_matches_bruteforce(shape):
    x = _rand(shape, 1)
    ref = dft.dft3_bruteforce(x)
    got = dft.fft3(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)) * 10


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 6, 6), (2, 3, 4)])
def test_inverse_matches_bruteforce(shape):
    X = _rand(shape, 2)
    ref = dft.dft3_bruteforce(X, sign=+1) / X.size
    got = dft.ifft3(X)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)) * 10


@pytest.mark.parametrize("n", [4, 6, 8, 12, 16])
def test_round_trip_and_parseval(n):
    x = _rand((n, n, n), 3)
    X = dft.fft3(x)
    assert np.allclose(dft.ifft3(X), x, rtol=0, atol=1e-12)
    assert np.isclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / x.size, rtol=1e-13)


def test_single_mode_is_a_delta():
    n = 6
    k0 = (1, 4, 3)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    f = np.exp(2j * np.pi * (k0[0] * z + k0[1] * y + k0[2] * x) / n)
    F = dft.fft3(f)
    expect = np.zeros_like(F)
    expect[k0] = n ** 3
    assert np.max(np.abs(F - expect)) < 1e-10


@pytest.mark.parametrize("n", [8, 12, 24])
def test_matches_library_fft(n):
    x = _rand((n, n, n), 4)
    assert np.allclose(dft.fft3(x), np.fft.fftn(x), rtol=0, atol=1e-10)
