"""Discrete Fourier transforms written out from their definition (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The prior covariance S of Sec. 2.2 is a convolution, so it is diagonal in the
Fourier basis.  The convention used throughout (the paper defers it to an
earlier work) is the unnormalised forward DFT

    X[k] = sum_r x[r] exp(-2 pi i k.r / n)

and the inverse divided by n^3.  Two implementations:

* `dft3_bruteforce` sums the definition over all n^3 x n^3 index pairs
  (tiny grids only); it is the pin for the other one.
* `fft3` / `ifft3` apply the 1D DFT matrix along each axis in turn.  The 3D
  DFT kernel exp(-2 pi i k.r/n) factorises over axes, so this is the same sum
  evaluated axis by axis; the matrix product is a library primitive.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """F[j, k] = exp(sign * 2 pi i (j k mod n) / n)."""
    j = np.arange(n)
    phase = np.mod(np.outer(j, j), n).astype(np.float64) * (2.0 * np.pi / n)
    return np.cos(phase) + 1j * sign * np.sin(phase)


def dft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Unnormalised 1D DFT of x along `axis` (no 1/n factor)."""
    n = x.shape[axis]
    F = dft_matrix(n, sign)
    xm = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    out = xm.reshape(-1, n) @ F
    return np.moveaxis(out.reshape(xm.shape), -1, axis)


def fft3(x: np.ndarray) -> np.ndarray:
    """Forward 3D DFT, unnormalised."""
    X = np.asarray(x, dtype=np.complex128)
    for ax in range(3):
        X = dft_axis(X, ax, -1)
    return X


def ifft3(X: np.ndarray) -> np.ndarray:
    """Inverse 3D DFT, divided by the number of cells."""
    x = np.asarray(X, dtype=np.complex128)
    for ax in range(3):
        x = dft_axis(x, ax, +1)
    return x / x.size


def dft3_bruteforce(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """The 3D DFT as one dense sum over all cell/mode pairs (O(N^2))."""
    x = np.asarray(x, dtype=np.complex128)
    nz, ny, nx = x.shape
    z, y, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                           indexing="ij")
    z, y, xx = z.ravel(), y.ravel(), xx.ravel()
    # phase[k, r] = 2 pi (kz z / nz + ky y / ny + kx x / nx)
    phase = 2.0 * np.pi * (np.outer(z, z) / nz + np.outer(y, y) / ny
                           + np.outer(xx, xx) / nx)
    E = np.exp(sign * 1j * phase)
    return (E @ x.ravel()).reshape(x.shape)
