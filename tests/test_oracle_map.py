"""Pins for the oracle's MAP solve and its implicit adjoint.

* Diagonal prior S_L = sigma^2 I (DC included): every cell decouples and
  Eq. (MAPLNUB) has the Lambert-W closed form, with the FFTs still active.
* Flat-prior limit (sigma^2 -> infinity): s* -> ln(N / (w nbar)), the
  inverse-weighting row of Table 1 (Sec. 4.1.1), for N > 0.
* Full prior: the objective is strictly convex, so the MAP is unique (same
  answer from different starts); with a flat prior on the mean the DC
  component of the gradient gives sum w nbar e^s* = sum N.
* Implicit adjoint: central finite differences in the counts and in ln A.
"""
import math

import numpy as np
import pytest

from oracle import plc
from paper_0911_1407_gb300 import mocks


def _const_table(n, box, sigma2):
    """Table with P = sigma2 L^3 / n^3, so lambda_k = sigma2 for every k."""
    kf = 2 * math.pi / box
    k = np.array([0.5 * kf, 2 * math.sqrt(3) * math.pi * n / box])
    return k, np.full(2, sigma2 * box ** 3 / n ** 3)


@pytest.mark.parametrize("n,sigma2,with_w", [(8, 1.5, False), (12, 0.7, True), (6, 4.0, True)])
def test_diagonal_prior_matches_lambert_w(n, sigma2, with_w):
    rng = np.random.default_rng(n)
    box = 60.0
    N = rng.poisson(3.0, size=(n, n, n))
    N.flat[0] = 40
    w = rng.uniform(0.1, 1.0, size=(n, n, n)) if with_w else None
    nbar, mu = 1.3, -0.5 * sigma2
    k, P = _const_table(n, box, sigma2)
    p = plc.make_problem(N, w, nbar, mu, n, box, k, P, inv_lambda_dc=1.0 / sigma2)
    res = plc.newton_krylov_map(p, tol=1e-13)
    assert res.converged
    exact = plc.map_closed_form_diagonal(N, w, nbar, mu, sigma2)
    err = np.abs(res.s - exact) / np.maximum(np.abs(exact), 1.0)
    assert err.max() <= 1e-11


def test_flat_prior_limit_is_inverse_weighting():
    n = 6
    rng = np.random.default_rng(11)
    N = rng.poisson(4.0, size=(n, n, n))
    w = rng.uniform(0.3, 1.0, size=(n, n, n))
    nbar, sigma2 = 2.0, 1e6
    k, P = _const_table(n, 30.0, sigma2)
    p = plc.make_problem(N, w, nbar, 0.0, n, 30.0, k, P, inv_lambda_dc=1.0 / sigma2)
    res = plc.newton_krylov_map(p, tol=1e-13, max_newton=200)
    assert res.converged
    pos = N > 0
    assert np.max(np.abs(res.s[pos] - np.log(N[pos] / (w[pos] * nbar)))) < 1e-4
    # empty cells are pushed far below every occupied level
    if np.any(~pos):
        assert res.s[~pos].max() < np.log(1.0 / (w.max() * nbar)) - 5


def _small_mock(n=16, selection="uniform", sigma=1.0, nbar=2.0):
    m = mocks.make_mock(mocks.small_spec(n, box=100.0, sigma_G=sigma, nbar=nbar,
                                         selection=selection, nbins=128))
    p = plc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    return m, p


@pytest.mark.parametrize("selection", ["uniform", "radial_masked"])
def test_full_prior_map_unique_and_conserves_mass(selection):
    m, p = _small_mock(selection=selection)
    a = plc.newton_krylov_map(p, tol=1e-12)
    assert a.converged and a.grad_rel < 1e-12
    D = p.wn * np.exp(a.s)
    assert abs(D.sum() - m.N.sum()) <= 1e-9 * m.N.sum()
    s0 = m.mu + 0.3 * np.random.default_rng(3).standard_normal(m.N.shape)
    b = plc.newton_krylov_map(p, s0=s0, tol=1e-12)
    assert b.converged
    assert np.max(np.abs(a.s - b.s) / np.maximum(np.abs(a.s), 1)) < 1e-9


def test_map_beats_inverse_weighting_on_truth():
    """Sanity, not parity: Sec. 4.1.2 correlation r against the true field."""
    m, p = _small_mock(n=24, sigma=1.0, nbar=1.0)
    a = plc.newton_krylov_map(p, tol=1e-8)
    d_true = np.exp(m.s_true) - 1
    d_map = np.exp(a.s) - 1
    d_iw = m.N / m.nbar - 1

    def r(a_, b_):
        return np.sum(a_ * b_) / math.sqrt(np.sum(a_ * a_) * np.sum(b_ * b_))
    assert r(d_map, d_true) > r(d_iw, d_true)


def test_vjp_matches_finite_differences():
    m, p = _small_mock(n=8, sigma=1.0, nbar=2.0)
    sol = plc.newton_krylov_map(p, tol=1e-14)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(m.N.shape)
    lam, vjp_lnA, _ = plc.map_vjp(sol.s, u, p, rtol=1e-13)
    # counts, as reals, along a random direction
    dN = rng.standard_normal(m.N.shape)
    eps = 1e-4
    sp = plc.newton_krylov_map(plc.Problem(m.N + eps * dN, p.w, p.nbar, p.mu, p.inv_lam), s0=sol.s, tol=1e-14).s
    sm = plc.newton_krylov_map(plc.Problem(m.N - eps * dN, p.w, p.nbar, p.mu, p.inv_lam), s0=sol.s, tol=1e-14).s
    fd = np.sum(u * (sp - sm)) / (2 * eps)
    assert abs(fd - np.sum(lam * dN)) <= 1e-6 * abs(fd)
    # amplitude of the power spectrum, in ln A
    def solve_scaled(f):
        pa = plc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab * f)
        return plc.newton_krylov_map(pa, s0=sol.s, tol=1e-14).s
    fdA = np.sum(u * (solve_scaled(math.exp(eps)) - solve_scaled(math.exp(-eps)))) / (2 * eps)
    assert abs(fdA - vjp_lnA) <= 1e-6 * abs(fdA)
