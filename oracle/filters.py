"""The paper's other density estimators on the same grid (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy, written
for a reader checking it against the paper.  Same conventions as plc.py
(prior eigenvalues 1/lambda_k on the full DFT grid, counts N, completeness
w, mean count nbar); here the signal is the overdensity delta itself, with
prior mean 0.

LSQ-Wiener filter, unity bias (Sec. 4.1.1, Eq. WF; Table 1, Gaussian prior
and Gaussian likelihood).  With the data vector delta_g^o = N / nbar - w
(Eq. datamodel) and the noise covariance diag(w / nbar) (Eq. noiseav),
W^T N^-1 W = diag(nbar w) and W^T N^-1 delta_g^o = N - nbar w, so

    (S^-1 + diag(nbar w)) delta = N - nbar w.

Gaussian prior and Poisson likelihood, unity bias (Sec. 2.2.2, Eq. MAPG;
gradient and Hessian of Sec. 3.1.1, where they are written multiplied by S).
The MAP minimises

    L_G(delta) = 1/2 delta^T S^-1 delta + sum_i [ nbar w_i (1 + delta_i) - N_i ln(1 + delta_i) ]
    g = S^-1 delta + nbar w - N / (1 + delta)
    H = S^-1 + diag(N / (1 + delta)^2)

on the set where 1 + delta_i > 0 for every cell with N_i > 0 (cells with
N_i = 0 carry no logarithm and may go below -1, the negative densities the
paper reports for this filter in Sec. 4.3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .dft import fft3, ifft3
from .plc import CGResult, Problem, apply_Sinv, pcg


# ---------------------------------------------------------------------------
# LSQ-Wiener filter
# ---------------------------------------------------------------------------

def wiener_lsq(p: Problem, rtol: float = 1e-13, maxit: int = 5000):
    """delta = (S^-1 + diag(nbar w))^-1 (N - nbar w) by Jacobi-preconditioned CG."""
    wn = p.wn * np.ones(p.N.shape)
    b = p.N.astype(np.float64) - wn
    mdiag = wn + float(np.mean(p.inv_lam))
    cg = pcg(lambda v: apply_Sinv(v, p.inv_lam) + wn * v, b, mdiag, rtol, maxit)
    return cg.x, cg


def wiener_closed_form_uniform(N, nbar: float, inv_lam) -> np.ndarray:
    """w = 1: S^-1 + nbar I is diagonal in Fourier space, so
    delta = IDFT( DFT(N - nbar) / (1/lambda_k + nbar) )."""
    b = np.asarray(N, dtype=np.float64) - nbar
    return ifft3(fft3(b) / (inv_lam + nbar)).real


def wiener_closed_form_diagonal(N, w, nbar: float, sigma2: float) -> np.ndarray:
    """S = sigma2 I: delta = (N - nbar w) / (1/sigma2 + nbar w), cell by cell."""
    N = np.asarray(N, dtype=np.float64)
    wn = nbar * (np.ones_like(N) if w is None else np.asarray(w, np.float64))
    return (N - wn) / (1.0 / sigma2 + wn)


# ---------------------------------------------------------------------------
# Gaussian prior, Poisson likelihood
# ---------------------------------------------------------------------------

def gauss_neg_log_posterior(delta: np.ndarray, p: Problem) -> float:
    """L_G(delta) (constants dropped); +inf outside the domain."""
    one = 1.0 + delta
    pos = p.N > 0
    if np.any(one[pos] <= 0.0):
        return math.inf
    prior = 0.5 * float(np.sum(delta * apply_Sinv(delta, p.inv_lam)))
    like = float(np.sum(p.wn * one)) - float(np.sum(p.N[pos] * np.log(one[pos])))
    return prior + like


def gauss_gradient(delta: np.ndarray, p: Problem) -> np.ndarray:
    """g = S^-1 delta + nbar w - N / (1 + delta)."""
    return apply_Sinv(delta, p.inv_lam) + p.wn - p.N / (1.0 + delta)


def gauss_diagonal(delta: np.ndarray, p: Problem) -> np.ndarray:
    """The likelihood's Hessian diagonal N / (1 + delta)^2."""
    return p.N / (1.0 + delta) ** 2


def gauss_hessvec(delta: np.ndarray, v: np.ndarray, p: Problem) -> np.ndarray:
    """H v = S^-1 v + diag(N / (1 + delta)^2) v."""
    return apply_Sinv(v, p.inv_lam) + gauss_diagonal(delta, p) * v


@dataclass
class GaussMapResult:
    delta: np.ndarray
    converged: bool
    newton_iters: int
    cg_iters: int
    grad_rel: float
    neg_logpost: float
    g0_norm: float
    history: list = field(default_factory=list)


def gauss_map(p: Problem, delta0: Optional[np.ndarray] = None, tol: float = 1e-12,
              max_newton: int = 100, max_cg: int = 1000, frac: float = 0.99,
              armijo_c: float = 1e-4, max_halvings: int = 30) -> GaussMapResult:
    """MAP of Eq. (MAPG) by inexact Newton-Krylov, as the lognormal MAP in
    plc.newton_krylov_map (CG forcing term, tau of Eq. New5, Armijo) with the
    step kept inside the domain: tau <= frac * min over cells with N > 0 and
    xi < 0 of (1 + delta) / (-xi) (fraction to the boundary) instead of a cap
    on max |tau xi|.  delta0 defaults to the prior mean 0."""
    delta = np.zeros(p.N.shape) if delta0 is None else np.array(delta0, dtype=np.float64)
    pos = p.N > 0
    g = gauss_gradient(delta, p)
    f = gauss_neg_log_posterior(delta, p)
    g0 = math.sqrt(float(np.sum(g * g)))
    gnorm, it, cg_total, hist = g0, 0, 0, []
    while True:
        rel = gnorm / g0 if g0 > 0 else 0.0
        if rel < tol:
            return GaussMapResult(delta, True, it, cg_total, rel, f, g0, hist)
        if it >= max_newton:
            return GaussMapResult(delta, False, it, cg_total, rel, f, g0, hist)
        eta = min(0.5, max(math.sqrt(rel), 0.3 * tol / rel))
        mdiag = gauss_diagonal(delta, p) + float(np.mean(p.inv_lam))
        cg = pcg(lambda v: gauss_hessvec(delta, v, p), -g, mdiag, eta, max_cg)
        cg_total += cg.iters
        xi = cg.x
        if cg.iters == 0:
            return GaussMapResult(delta, rel < tol, it, cg_total, rel, f, g0, hist)
        xg = float(np.sum(xi * g))
        xHx = float(np.sum(xi * gauss_hessvec(delta, xi, p)))
        tau = -xg / xHx                                  # Eq. (New5)
        toward = pos & (xi < 0.0)
        if np.any(toward):
            tau = min(tau, frac * float(np.min((1.0 + delta[toward]) / -xi[toward])))
        scale = float(np.sum(p.wn * np.abs(1.0 + delta))) + abs(f)
        for _ in range(max_halvings):
            f_try = gauss_neg_log_posterior(delta + tau * xi, p)
            if f_try <= f + armijo_c * tau * xg or -tau * xg < 1e-13 * scale:
                break
            tau *= 0.5
        delta = delta + tau * xi
        g = gauss_gradient(delta, p)
        f = gauss_neg_log_posterior(delta, p)
        gnorm = math.sqrt(float(np.sum(g * g)))
        it += 1
        hist.append((it, gnorm / g0, f, cg.iters, tau))


def gauss_closed_form_diagonal(N, w, nbar: float, sigma2: float) -> np.ndarray:
    """S = sigma2 I: cell by cell, delta / sigma2 + nbar w - N / (1 + delta) = 0,
    i.e. delta^2 + (1 + a) delta + a - sigma2 N = 0 with a = sigma2 nbar w.
    For N > 0 the root with 1 + delta > 0 is
    delta = (-(1 + a) + sqrt((1 - a)^2 + 4 sigma2 N)) / 2; for N = 0 the
    objective is the parabola delta^2 / (2 sigma2) + nbar w delta, so delta = -a."""
    N = np.asarray(N, dtype=np.float64)
    a = sigma2 * nbar * (np.ones_like(N) if w is None else np.asarray(w, np.float64))
    root = 0.5 * (-(1.0 + a) + np.sqrt((1.0 - a) ** 2 + 4.0 * sigma2 * N))
    return np.where(N > 0, root, -a)
