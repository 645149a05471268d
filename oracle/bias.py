"""Lognormal prior, Poisson likelihood, linear bias (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy.

Sec. 2.4.1: the galaxy field is a linear transform of the matter field,
delta_g = B delta_M, with B a convolution whose Fourier transform is the
bias b(|k|) (Sec. 2.2.1: b = sqrt(P_g / P_M)).  With s = ln(1 + delta_M) and
u = 1 + B(e^s - 1) the negative log posterior is

    L(s) = 1/2 (s - mu)^T S^-1 (s - mu) + sum_i [ nbar w_i u_i - N_i ln u_i ]

(defined where u_i > 0 for every cell with N_i > 0), whose gradient is the
linear-bias MAP equation of Sec. 2.4.1 (B symmetric):

    g = S^-1 (s - mu) + e^s . B(nbar w - N / u)

and whose Hessian is

    H = S^-1 + diag(e^s . B(nbar w - N / u)) + diag(e^s) B diag(N / u^2) B diag(e^s).

b(|k|) is tabulated like P(k) (linear in (ln k, ln b) between table points);
the DC mode has its own bias b_dc.  With b = 1 everywhere this is the
unity-bias problem of plc.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .dft import fft3, ifft3
from .plc import Problem, apply_Sinv, interp_pk, mode_wavenumbers, pcg


def bias_multipliers(n: int, box: float, k_tab, b_tab, b_dc: float = 1.0) -> np.ndarray:
    """b_k on the full n^3 DFT grid, linear in (ln k, ln b) inside the table."""
    kk = mode_wavenumbers(n, box)
    kk_nz = kk.copy()
    kk_nz[0, 0, 0] = k_tab[0]
    b = interp_pk(kk_nz, k_tab, b_tab)
    b[0, 0, 0] = b_dc
    return b


def apply_B(x: np.ndarray, bk: np.ndarray) -> np.ndarray:
    return ifft3(fft3(x) * bk).real


@dataclass
class BiasProblem:
    p: Problem          # counts, selection, nbar, mu and S^-1
    bk: np.ndarray      # b_k on the full grid


def galaxy_density(s: np.ndarray, q: BiasProblem) -> np.ndarray:
    """u = 1 + B(e^s - 1)."""
    return 1.0 + apply_B(np.expm1(s), q.bk)


def bias_neg_log_posterior(s: np.ndarray, q: BiasProblem) -> float:
    p = q.p
    u = galaxy_density(s, q)
    occ = p.N > 0
    if np.any(u[occ] <= 0.0):
        return math.inf
    prior = 0.5 * float(np.sum((s - p.mu) * apply_Sinv(s - p.mu, p.inv_lam)))
    return prior + float(np.sum(p.wn * u)) - float(np.sum(p.N[occ] * np.log(u[occ])))


def bias_gradient(s: np.ndarray, q: BiasProblem) -> np.ndarray:
    p = q.p
    u = galaxy_density(s, q)
    return apply_Sinv(s - p.mu, p.inv_lam) + np.exp(s) * apply_B(p.wn - p.N / u, q.bk)


def bias_hessvec(s: np.ndarray, v: np.ndarray, q: BiasProblem) -> np.ndarray:
    p = q.p
    e = np.exp(s)
    u = galaxy_density(s, q)
    first = e * apply_B(p.wn - p.N / u, q.bk)
    second = e * apply_B(p.N / u ** 2 * apply_B(e * v, q.bk), q.bk)
    return apply_Sinv(v, p.inv_lam) + first * v + second


@dataclass
class BiasMapResult:
    s: np.ndarray
    converged: bool
    newton_iters: int
    cg_iters: int
    grad_rel: float
    neg_logpost: float
    g0_norm: float
    history: list = field(default_factory=list)


def bias_map(q: BiasProblem, s0: Optional[np.ndarray] = None, tol: float = 1e-12,
             max_newton: int = 200, max_cg: int = 1000, step_cap: float = 2.0,
             armijo_c: float = 1e-4, max_halvings: int = 40) -> BiasMapResult:
    """Newton-Krylov MAP as plc.newton_krylov_map (CG forcing term, tau of
    Eq. New5, max |tau xi| <= step_cap, Armijo) with the exact Hessian; CG
    stops at negative curvature (keeping the iterate so far, or the
    preconditioned gradient step if that happens at once).  Trial points
    outside the domain have L = +inf and are halved.  s0 defaults to 0
    (delta_M = 0, so u = 1 inside the domain whatever b is)."""
    p = q.p
    s = np.zeros(p.N.shape) if s0 is None else np.array(s0, dtype=np.float64)
    g = bias_gradient(s, q)
    f = bias_neg_log_posterior(s, q)
    g0 = math.sqrt(float(np.sum(g * g)))
    gnorm, it, cg_total, hist = g0, 0, 0, []
    while True:
        rel = gnorm / g0 if g0 > 0 else 0.0
        if rel < tol:
            return BiasMapResult(s, True, it, cg_total, rel, f, g0, hist)
        if it >= max_newton:
            return BiasMapResult(s, False, it, cg_total, rel, f, g0, hist)
        eta = min(0.5, max(math.sqrt(rel), 0.3 * tol / rel))
        u = galaxy_density(s, q)
        mdiag = np.abs(np.exp(s) * apply_B(p.wn - p.N / u, q.bk)) + np.exp(2 * s) * p.N / u ** 2 \
            + float(np.mean(p.inv_lam))
        cg = pcg(lambda v: bias_hessvec(s, v, q), -g, mdiag, eta, max_cg)
        cg_total += cg.iters
        xi = cg.x if cg.iters > 0 else -g / mdiag
        xg = float(np.sum(xi * g))
        xHx = float(np.sum(xi * bias_hessvec(s, xi, q)))
        tau = -xg / xHx if xHx > 0 else 1.0
        xmax = float(np.max(np.abs(xi)))
        if tau * xmax > step_cap:
            tau = step_cap / xmax
        scale = float(np.sum(p.wn * np.abs(u))) + abs(f)
        for _ in range(max_halvings):
            f_try = bias_neg_log_posterior(s + tau * xi, q)
            if f_try <= f + armijo_c * tau * xg or -tau * xg < 1e-13 * scale:
                break
            tau *= 0.5
        s = s + tau * xi
        g = bias_gradient(s, q)
        f = bias_neg_log_posterior(s, q)
        gnorm = math.sqrt(float(np.sum(g * g)))
        it += 1
        hist.append((it, gnorm / g0, f, cg.iters, tau))


def bias_closed_form_cell(N: float, wn: float, mu: float, sigma2: float, b: float) -> float:
    """Diagonal prior S = sigma2 I and constant bias b (DC included), one cell:
    (s - mu)/sigma2 + b e^s (wn - N / (1 + b (e^s - 1))) = 0, solved by
    bisection on the interval where 1 + b(e^s - 1) > 0 (N > 0) -- a brute
    force reference for the coupled solve."""
    def h(s):
        u = 1.0 + b * math.expm1(s)
        return (s - mu) / sigma2 + b * math.exp(s) * (wn - (N / u if N > 0 else 0.0))
    lo = math.log1p(-1.0 / b) + 1e-15 if (N > 0 and b > 1.0) else -60.0
    hi = 60.0
    while h(lo) > 0:      # N = 0 or b <= 1: widen below
        lo -= 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if h(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)
