"""Poisson-lognormal MAP: objective, derivatives and Newton-Krylov (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy, written
for a reader checking it against the paper, not for speed.

Notation (paper, Sec. 2-3, unity bias):
  s        log-density ln(1 + delta) per cell (Sec. 2.3)
  N        observed counts N^o_g (Sec. 2.1)
  w        completeness per cell; None means w = 1
  nbar     mean count N-bar_g (Sec. 2.1, definition of <N>)
  mu       constant prior mean (Sec. 2.3, Eq. mu)
  S^-1     inverse prior covariance, a convolution: diagonal in Fourier space
           with eigenvalue 1/lambda_k (Sec. 2.2)

Readings of points the paper leaves open:
  * lambda_k = P(|k|) n^3 / L^3 under the unnormalised forward DFT;
    |k| = (2 pi / L) |m|, m in [-n/2, n/2) per axis.
  * P between table points is linear in (ln k, ln P).
  * The DC mode has no power (P(0) = 0); its inverse eigenvalue is an input,
    0 by default (a flat prior on the mean).
  * The objective drops the constants -N ln(w nbar) + ln N! of the likelihood.

Objective (negative log posterior, Sec. 2.1 likelihood and Sec. 2.3 prior):
    L(s) = 1/2 (s - mu)^T S^-1 (s - mu) + sum_i [ w_i nbar e^{s_i} - N_i s_i ]
Gradient (Sec. 3.1.2):  g = S^-1 (s - mu) + diag(nbar w) e^s - N
Hessian  (Sec. 3.1.2):  H = S^-1 + diag(nbar w e^s)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .dft import fft3, ifft3
from .lambertw import lambertw_from_log


# ---------------------------------------------------------------------------
# Prior spectrum (Sec. 2.2: S is a convolution whose Fourier transform is P)
# ---------------------------------------------------------------------------

def mode_wavenumbers(n: int, box: float) -> np.ndarray:
    """|k| for every mode of the full n^3 grid, [kz][ky][kx] order."""
    m = np.arange(n)
    m = np.where(m < (n + 1) // 2, m, m - n).astype(np.float64)
    m2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    return (2.0 * np.pi / box) * np.sqrt(m2)


def interp_pk(k: np.ndarray, k_tab: np.ndarray, P_tab: np.ndarray) -> np.ndarray:
    """P(k) by linear interpolation in (ln k, ln P) inside the table."""
    k_tab = np.asarray(k_tab, dtype=np.float64)
    P_tab = np.asarray(P_tab, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    if np.any(k < k_tab[0]) or np.any(k > k_tab[-1]):
        raise ValueError("power-spectrum table does not cover the grid's modes")
    j = np.clip(np.searchsorted(k_tab, k, side="right") - 1, 0, k_tab.size - 2)
    lk0, lk1 = np.log(k_tab[j]), np.log(k_tab[j + 1])
    lp0, lp1 = np.log(P_tab[j]), np.log(P_tab[j + 1])
    t = (np.log(k) - lk0) / (lk1 - lk0)
    return np.exp(lp0 + t * (lp1 - lp0))


def inverse_eigenvalues(n: int, box: float, k_tab, P_tab,
                        inv_lambda_dc: float = 0.0) -> np.ndarray:
    """1/lambda_k on the full n^3 DFT grid, lambda_k = P(|k|) n^3 / L^3."""
    kk = mode_wavenumbers(n, box)
    kk_nz = kk.copy()
    kk_nz[0, 0, 0] = k_tab[0]           # placeholder, overwritten below
    lam = interp_pk(kk_nz, k_tab, P_tab) * (n ** 3 / box ** 3)
    inv = 1.0 / lam
    inv[0, 0, 0] = inv_lambda_dc
    return inv


@dataclass
class Problem:
    """Inputs of one MAP solve (the paper's N, w, nbar, mu and S)."""
    N: np.ndarray
    w: Optional[np.ndarray]
    nbar: float
    mu: float
    inv_lam: np.ndarray                 # 1/lambda_k, full grid

    @property
    def wn(self) -> np.ndarray | float:
        """nbar * w per cell (a scalar when w = 1)."""
        return self.nbar if self.w is None else self.nbar * self.w


def make_problem(N, w, nbar, mu, n, box, k_tab, P_tab,
                 inv_lambda_dc: float = 0.0) -> Problem:
    return Problem(np.asarray(N), None if w is None else np.asarray(w, float),
                   float(nbar), float(mu),
                   inverse_eigenvalues(n, box, k_tab, P_tab, inv_lambda_dc))


# ---------------------------------------------------------------------------
# Operators
# ---------------------------------------------------------------------------

def apply_Sinv(x: np.ndarray, inv_lam: np.ndarray) -> np.ndarray:
    """S^-1 x = IDFT( DFT(x) / lambda_k ) (convolution theorem, Sec. 2.2)."""
    return ifft3(fft3(x) * inv_lam).real


def diagonal(s: np.ndarray, p: Problem) -> np.ndarray:
    """D = nbar w e^s, the expected count per cell (Sec. 2.1, 3.1.2)."""
    return p.wn * np.exp(s)


def neg_log_posterior(s: np.ndarray, p: Problem) -> float:
    """-ln P(s|N) up to constants: prior (Sec. 2.3) plus likelihood (Sec. 2.1)."""
    r = s - p.mu
    prior = 0.5 * float(np.sum(r * apply_Sinv(r, p.inv_lam)))
    like = float(np.sum(diagonal(s, p) - p.N * s))
    return prior + like


def gradient(s: np.ndarray, p: Problem) -> np.ndarray:
    """g = S^-1 (s - mu) + diag(nbar w) e^s - N (Sec. 3.1.2)."""
    return apply_Sinv(s - p.mu, p.inv_lam) + diagonal(s, p) - p.N


def hessvec(s: np.ndarray, v: np.ndarray, p: Problem) -> np.ndarray:
    """H v = S^-1 v + diag(nbar w e^s) v (Sec. 3.1.2)."""
    return apply_Sinv(v, p.inv_lam) + diagonal(s, p) * v


def jacobi_diagonal(s: np.ndarray, p: Problem) -> np.ndarray:
    """diag(H) = nbar w e^s + (S^-1)_ii, where (S^-1)_ii = mean_k 1/lambda_k."""
    return diagonal(s, p) + float(np.mean(p.inv_lam))


# ---------------------------------------------------------------------------
# Solvers
# ---------------------------------------------------------------------------

@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    rel_res: float
    breakdown: bool = False


def pcg(apply_H, b: np.ndarray, mdiag: Optional[np.ndarray], rtol: float,
        maxit: int) -> CGResult:
    """Preconditioned conjugate gradients for H x = b from x = 0.

    Stops when ||r|| <= rtol ||b||; the preconditioner is diag(mdiag)^-1
    (identity when mdiag is None).
    """
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = math.sqrt(float(np.sum(b * b)))
    if bnorm == 0.0:
        return CGResult(x, 0, 0.0)
    z = r / mdiag if mdiag is not None else r.copy()
    pdir = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    rnorm = bnorm
    while it < maxit and rnorm > rtol * bnorm:
        Hp = apply_H(pdir)
        pHp = float(np.sum(pdir * Hp))
        if not pHp > 0.0:
            return CGResult(x, it, rnorm / bnorm, breakdown=True)
        alpha = rz / pHp
        x += alpha * pdir
        r -= alpha * Hp
        it += 1
        rnorm = math.sqrt(float(np.sum(r * r)))
        z = r / mdiag if mdiag is not None else r.copy()
        rz_new = float(np.sum(r * z))
        beta = rz_new / rz
        rz = rz_new
        pdir = z + beta * pdir
    return CGResult(x, it, rnorm / bnorm)


@dataclass
class MapResult:
    s: np.ndarray
    converged: bool
    newton_iters: int
    cg_iters: int
    grad_rel: float
    neg_logpost: float
    g0_norm: float
    history: list = field(default_factory=list)


def newton_krylov_map(p: Problem, s0: Optional[np.ndarray] = None,
                      tol: float = 1e-12, max_newton: int = 100,
                      max_cg: int = 500, g0_norm: float = 0.0,
                      step_cap: float = 2.0, armijo_c: float = 1e-4,
                      max_halvings: int = 30) -> MapResult:
    """MAP of the Poisson-lognormal posterior by inexact Newton-Krylov.

    Sec. 3.1: x^{j+1} = x^j + tau^j xi^j with tau from Eq. (New5),
    tau = -xi^T grad Q / (xi^T H xi).  The paper leaves the search vector xi to
    earlier work; here xi solves H xi = -g by Jacobi-preconditioned CG to a
    relative residual eta = min(0.5, max(sqrt(rel), 0.3 tol / rel)),
    rel = ||g|| / ||g0|| (superlinear, without solving past what the stop
    test needs).  The step is capped so that max |tau xi| <= step_cap, then
    halved until the Armijo condition L(s + tau xi) <= L(s) + c tau xi^T g
    holds (or the predicted decrease is below the rounding level of L).  Stops when ||g|| / ||g0|| < tol, with
    g0 = g(s0) unless g0_norm is given.  s0 defaults to mu.
    """
    shape = p.N.shape
    s = np.full(shape, p.mu, dtype=np.float64) if s0 is None else np.array(s0, dtype=np.float64)
    g = gradient(s, p)
    f = neg_log_posterior(s, p)
    gnorm = math.sqrt(float(np.sum(g * g)))
    g0 = g0_norm if g0_norm > 0.0 else gnorm
    hist = [(0, gnorm / g0, f)]
    cg_total = 0
    it = 0
    while True:
        rel = gnorm / g0 if g0 > 0 else 0.0
        if rel < tol:
            return MapResult(s, True, it, cg_total, rel, f, g0, hist)
        if it >= max_newton:
            return MapResult(s, False, it, cg_total, rel, f, g0, hist)
        eta = min(0.5, max(math.sqrt(rel), 0.3 * tol / rel))
        mdiag = jacobi_diagonal(s, p)
        cg = pcg(lambda v: hessvec(s, v, p), -g, mdiag, eta, max_cg)
        cg_total += cg.iters
        xi = cg.x
        if cg.iters == 0:                      # nothing to do (g = 0)
            return MapResult(s, rel < tol, it, cg_total, rel, f, g0, hist)
        xg = float(np.sum(xi * g))
        xHx = float(np.sum(xi * hessvec(s, xi, p)))
        tau = -xg / xHx                         # Eq. (New5)
        xmax = float(np.max(np.abs(xi)))
        if tau * xmax > step_cap:
            tau = step_cap / xmax
        # rounding level of L: its terms' magnitudes times a few ulps
        scale = float(np.sum(diagonal(s, p) + np.abs(p.N * s))) + abs(f)
        for _ in range(max_halvings):
            f_try = neg_log_posterior(s + tau * xi, p)
            if f_try <= f + armijo_c * tau * xg or -tau * xg < 1e-13 * scale:
                break
            tau *= 0.5
        s = s + tau * xi
        g = gradient(s, p)
        f = neg_log_posterior(s, p)
        gnorm = math.sqrt(float(np.sum(g * g)))
        it += 1
        hist.append((it, gnorm / g0, f, cg.iters, tau))


def map_vjp(s_map: np.ndarray, u: np.ndarray, p: Problem, rtol: float = 1e-12,
            max_cg: int = 2000):
    """Implicit adjoint of the MAP (implicit-function theorem on g(s*) = 0).

    With g(s*; N, alpha) = 0 and dg/dN = -I, ds*/dN = H^-1.  Scaling every
    non-DC prior eigenvalue lambda_k -> alpha lambda_k gives
    dg/d(alpha) = -S^-1_{k!=0} (s - mu) at alpha = 1, so
    ds*/d(ln A) = H^-1 S^-1_{k!=0} (s* - mu).  For a cotangent u, with
    lam = H^-1 u (one CG solve; H is symmetric):
        vjp_N   = lam
        vjp_lnA = lam^T S^-1_{k!=0} (s* - mu)
    """
    mdiag = jacobi_diagonal(s_map, p)
    cg = pcg(lambda v: hessvec(s_map, v, p), u, mdiag, rtol, max_cg)
    lam = cg.x
    inv_nodc = p.inv_lam.copy()
    inv_nodc[0, 0, 0] = 0.0
    vjp_lnA = float(np.sum(lam * apply_Sinv(s_map - p.mu, inv_nodc)))
    return lam, vjp_lnA, cg


def map_closed_form_diagonal(N, w, nbar: float, mu: float, sigma2: float):
    """MAP for a diagonal prior S_L = sigma2 I (Eq. MAPLNUB cell by cell).

    (s - mu)/sigma2 + w nbar e^s = N  =>  s = mu + sigma2 N - W(x),
    x = sigma2 w nbar exp(mu + sigma2 N); W is evaluated from ln x.
    """
    N = np.asarray(N, dtype=np.float64)
    wn = nbar * (np.ones_like(N) if w is None else np.asarray(w, np.float64))
    with np.errstate(divide="ignore"):
        log_x = np.log(sigma2 * wn) + mu + sigma2 * N
    return mu + sigma2 * N - lambertw_from_log(log_x)
