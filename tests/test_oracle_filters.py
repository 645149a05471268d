"""Pins for the oracle's LSQ-Wiener filter and Gaussian-prior MAP.

LSQ-Wiener (Sec. 4.1.1, Eq. WF, Table 1):
* diagonal prior S = sigma^2 I (DC included): every cell decouples,
  delta = (N - nbar w) / (1/sigma^2 + nbar w), with the FFTs active;
* w = 1: S^-1 + nbar I is diagonal in Fourier space (the textbook Wiener
  filter), solved without CG by one forward and one inverse DFT;
* flat-prior limit: delta -> N / (nbar w) - 1, the inverse-weighting
  estimator (Table 1, flat prior).
Gaussian prior, Poisson likelihood (Eq. MAPG, Sec. 3.1.1):
* gradient and Hessian against central finite differences of the objective;
* diagonal prior: the per-cell quadratic has the closed-form root;
* the MAP satisfies the paper's own form of the MAP equation,
  delta = S (N / (1 + delta) - nbar w), applied with S (not S^-1).
"""
import math

import numpy as np
import pytest

from oracle import filters, plc
from tests.test_oracle_map import _const_table


def _problem(n, box, rng, with_w, nbar=1.4, dc=0.0, sigma=None, N_mean=2.5):
    N = rng.poisson(N_mean, size=(n, n, n))
    N.flat[3] = 30
    w = rng.uniform(0.1, 1.0, size=(n, n, n)) if with_w else None
    if sigma is None:
        from tests.gpu_util import pk_table_for
        k, P = pk_table_for(n, box, seed=n)
    else:
        k, P = _const_table(n, box, sigma)
    return plc.make_problem(N, w, nbar, 0.0, n, box, k, P, inv_lambda_dc=dc)


@pytest.mark.parametrize("n,sigma2,with_w", [(8, 1.5, True), (6, 0.4, False), (12, 3.0, True)])
def test_lsq_diagonal_prior(n, sigma2, with_w):
    rng = np.random.default_rng(n)
    p = _problem(n, 50.0, rng, with_w, sigma=sigma2, dc=1.0 / sigma2)
    delta, cg = filters.wiener_lsq(p, rtol=1e-14)
    exact = filters.wiener_closed_form_diagonal(p.N, p.w, p.nbar, sigma2)
    assert np.max(np.abs(delta - exact)) <= 1e-12 * np.max(np.abs(exact))


@pytest.mark.parametrize("n,dc", [(8, 0.0), (12, 0.3), (6, 0.0)])
def test_lsq_uniform_selection_is_fourier_diagonal(n, dc):
    rng = np.random.default_rng(100 + n)
    p = _problem(n, 7.0 * n, rng, False, dc=dc)
    delta, cg = filters.wiener_lsq(p, rtol=1e-14)
    exact = filters.wiener_closed_form_uniform(p.N, p.nbar, p.inv_lam)
    assert np.max(np.abs(delta - exact)) <= 1e-11 * np.max(np.abs(exact))


def test_lsq_flat_prior_limit_is_inverse_weighting():
    rng = np.random.default_rng(5)
    p = _problem(6, 30.0, rng, True, sigma=1e8, dc=1e-8)
    delta, _ = filters.wiener_lsq(p, rtol=1e-15)
    iw = p.N / (p.nbar * p.w) - 1.0
    assert np.max(np.abs(delta - iw)) <= 1e-6 * np.max(np.abs(iw))


def test_gauss_gradient_and_hessian_finite_differences():
    rng = np.random.default_rng(7)
    p = _problem(8, 60.0, rng, True, dc=0.2)
    delta = rng.uniform(-0.6, 1.5, size=p.N.shape)   # inside the domain
    d = rng.standard_normal(p.N.shape)
    h = 1e-6
    fd = (filters.gauss_neg_log_posterior(delta + h * d, p)
          - filters.gauss_neg_log_posterior(delta - h * d, p)) / (2 * h)
    an = float(np.sum(filters.gauss_gradient(delta, p) * d))
    assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0)
    v = rng.standard_normal(p.N.shape)
    fdh = (filters.gauss_gradient(delta + h * v, p) - filters.gauss_gradient(delta - h * v, p)) / (2 * h)
    hv = filters.gauss_hessvec(delta, v, p)
    assert np.max(np.abs(fdh - hv)) <= 1e-6 * np.max(np.abs(hv))
    u = rng.standard_normal(p.N.shape)
    assert abs(np.sum(u * filters.gauss_hessvec(delta, v, p))
               - np.sum(v * filters.gauss_hessvec(delta, u, p))) <= 1e-12 * np.sum(np.abs(u * v)) * 100


@pytest.mark.parametrize("n,sigma2,with_w", [(8, 1.5, True), (6, 4.0, False), (12, 0.3, True)])
def test_gauss_map_diagonal_prior_closed_form(n, sigma2, with_w):
    rng = np.random.default_rng(20 + n)
    p = _problem(n, 40.0, rng, with_w, sigma=sigma2, dc=1.0 / sigma2)
    res = filters.gauss_map(p, tol=1e-13)
    assert res.converged
    exact = filters.gauss_closed_form_diagonal(p.N, p.w, p.nbar, sigma2)
    err = np.abs(res.delta - exact) / np.maximum(np.abs(exact), 1.0)
    assert err.max() <= 1e-11
    assert np.all(1.0 + res.delta[p.N > 0] > 0.0)


def test_gauss_map_satisfies_the_printed_map_equation():
    """Eq. (MAPG): delta = S (N / (1 + delta) - nbar w), with S applied as
    IDFT(lambda_k DFT(.)); a finite DC eigenvalue so that S exists."""
    rng = np.random.default_rng(9)
    p = _problem(12, 90.0, rng, True, dc=0.5)
    res = filters.gauss_map(p, tol=1e-13)
    assert res.converged
    lam = 1.0 / p.inv_lam
    from oracle.dft import fft3, ifft3
    rhs = ifft3(lam * fft3(p.N / (1.0 + res.delta) - p.wn)).real
    assert np.max(np.abs(res.delta - rhs)) <= 1e-9 * max(np.max(np.abs(res.delta)), 1.0)
    # cells without galaxies may sit below delta = -1 (no logarithmic barrier)
    assert np.all(1.0 + res.delta[p.N > 0] > 0.0)
