"""Principal-branch Lambert W for non-negative arguments (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

W(x) is the w >= 0 with w e^w = x.  It gives the MAP of Eq. (MAPLNUB) in
closed form when the prior is diagonal (S_L = sigma^2 I): each cell then
solves (s - mu)/sigma^2 + w nbar e^s = N on its own, whose solution is
s = mu + sigma^2 N - W(sigma^2 w nbar exp(mu + sigma^2 N)).

The argument can overflow a double (sigma^2 N of several hundred), so the
function takes ln x.  Two iterations, both from Corless et al. (1996):
  * ln x <= 1: Halley's method on f(w) = w e^w - x;
  * ln x  > 1: Newton's method on f(w) = w + ln w - ln x (same root for w>0).
"""
from __future__ import annotations

import math

import numpy as np


def _w_scalar_from_log(lx: float) -> float:
    if lx == -math.inf:
        return 0.0
    if lx <= 1.0:
        x = math.exp(lx)
        w = math.log1p(x)              # W(x) <= ln(1 + x), a safe start
        for _ in range(100):
            ew = math.exp(w)
            f = w * ew - x
            denom = ew * (w + 1.0) - (w + 2.0) * f / (2.0 * w + 2.0)
            step = f / denom
            w -= step
            if abs(step) <= 4e-16 * max(abs(w), 1e-300):
                break
        return w
    w = lx - math.log(lx) if lx > 1.5 else 1.0
    for _ in range(100):
        f = w + math.log(w) - lx
        step = f / (1.0 + 1.0 / w)
        w -= step
        if abs(step) <= 4e-16 * abs(w):
            break
    return w


def lambertw_from_log(log_x) -> np.ndarray:
    """W(x) given ln x (elementwise); ln x = -inf means x = 0 and W = 0."""
    lx = np.asarray(log_x, dtype=np.float64)
    out = np.empty(lx.shape, dtype=np.float64)
    flat_in, flat_out = lx.ravel(), out.ravel()
    for i in range(flat_in.size):
        flat_out[i] = _w_scalar_from_log(float(flat_in[i]))
    return out


def lambertw(x) -> np.ndarray:
    """W(x) for x >= 0."""
    x = np.asarray(x, dtype=np.float64)
    if np.any(x < 0):
        raise ValueError("lambertw: only x >= 0 is supported")
    with np.errstate(divide="ignore"):
        return lambertw_from_log(np.log(x))
