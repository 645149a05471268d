"""Quality measures and matter statistics of a reconstruction (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy.

* Correlation coefficient between a reconstruction and the matter field
  (Sec. 4.1.2): r(a, b) = sum a b / (sqrt(sum a^2) sqrt(sum b^2)).
* Euclidean distance (Sec. 4.1.2, Eq. enseres):
  D_Euc(a, b) = sqrt(mean((a - b)^2)).
* Gaussian smoothing on the periodic grid (Sec. 4.3.3): convolution with a
  normalised Gaussian of radius r_S, i.e. multiplication of every Fourier
  mode by exp(-|k|^2 r_S^2 / 2), |k| = (2 pi / L) |m|, m in [-n/2, n/2).
* Matter statistics of ln(1 + delta) (Sec. 4.3.3): a histogram on fixed
  bins and the sample moments, skewness and excess kurtosis (the paper
  defers their formulas to earlier work; these are the standard population
  moments m_k = mean((x - mean)^k), skewness m_3 / m_2^(3/2), excess
  kurtosis m_4 / m_2^2 - 3), over the cells with 1 + delta > 0.
"""
from __future__ import annotations

import math

import numpy as np

from .dft import fft3, ifft3
from .plc import mode_wavenumbers


def correlation(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.sum(a * b) / (math.sqrt(float(np.sum(a * a))) * math.sqrt(float(np.sum(b * b)))))


def euclidean_distance(a: np.ndarray, b: np.ndarray) -> float:
    return math.sqrt(float(np.mean((a - b) ** 2)))


def gaussian_smooth(x: np.ndarray, box: float, radius: float) -> np.ndarray:
    n = x.shape[0]
    k = mode_wavenumbers(n, box)
    return ifft3(fft3(x) * np.exp(-0.5 * (k * radius) ** 2)).real


def log_density_stats(delta: np.ndarray, lo: float, width: float, nbins: int):
    """Histogram of x = ln(1 + delta) on bins [lo + j width, lo + (j+1) width),
    j < nbins (values outside count as below / above), and the moments of x
    over the cells with 1 + delta > 0.  Returns (counts, below, above,
    invalid, mean, variance, skewness, excess kurtosis)."""
    valid = 1.0 + delta > 0.0
    x = np.log(1.0 + delta[valid])
    j = np.floor((x - lo) / width).astype(np.int64)
    below = int(np.sum(j < 0))
    above = int(np.sum(j >= nbins))
    inside = j[(j >= 0) & (j < nbins)]
    counts = np.bincount(inside, minlength=nbins).astype(np.int64)
    mean = float(np.mean(x))
    d = x - mean
    m2, m3, m4 = float(np.mean(d ** 2)), float(np.mean(d ** 3)), float(np.mean(d ** 4))
    return counts, below, above, int(np.sum(~valid)), mean, m2, m3 / m2 ** 1.5, m4 / m2 ** 2 - 3.0
