"""Pins for the oracle's linear-bias lognormal MAP (Sec. 2.4.1).

* b = 1 everywhere: the problem is the unity-bias one, so the MAP equals
  plc.newton_krylov_map's (unique minimiser).
* Diagonal prior and constant bias (DC included): the cells decouple; each
  is a one-dimensional root found by bisection (brute force).
* Gradient and Hessian against central finite differences.
"""
import math

import numpy as np
import pytest

from oracle import bias, plc
from tests.test_oracle_map import _const_table


def _bias_table(n, box, b0, slope=0.0):
    kf = 2 * math.pi / box
    k = np.exp(np.linspace(math.log(0.5 * kf), math.log(2 * math.sqrt(3) * math.pi * n / box), 16))
    return k, b0 * (k / k[0]) ** slope


def _problem(n, box, rng, with_w, sigma=None, dc=0.0, nbar=1.3, mu=-0.4):
    N = rng.poisson(2.0, size=(n, n, n))
    N.flat[5] = 25
    w = rng.uniform(0.2, 1.0, size=(n, n, n)) if with_w else None
    if sigma is None:
        from tests.gpu_util import pk_table_for
        k, P = pk_table_for(n, box, seed=n)
    else:
        k, P = _const_table(n, box, sigma)
    return plc.make_problem(N, w, nbar, mu, n, box, k, P, inv_lambda_dc=dc)


def test_unit_bias_is_the_unity_bias_map():
    rng = np.random.default_rng(1)
    n, box = 8, 50.0
    p = _problem(n, box, rng, True, dc=0.3)
    kb, b = _bias_table(n, box, 1.0)
    q = bias.BiasProblem(p, bias.bias_multipliers(n, box, kb, b, 1.0))
    rb = bias.bias_map(q, tol=1e-13)
    ru = plc.newton_krylov_map(p, tol=1e-13)
    assert rb.converged and ru.converged
    assert np.max(np.abs(rb.s - ru.s) / np.maximum(np.abs(ru.s), 1.0)) <= 1e-10


@pytest.mark.parametrize("b0,sigma2", [(0.8, 1.2), (1.3, 0.7)])
def test_constant_bias_diagonal_prior_by_bisection(b0, sigma2):
    rng = np.random.default_rng(int(b0 * 10))
    n, box = 6, 30.0
    p = _problem(n, box, rng, True, sigma=sigma2, dc=1.0 / sigma2)
    kb, b = _bias_table(n, box, b0)
    q = bias.BiasProblem(p, bias.bias_multipliers(n, box, kb, b, b0))
    res = bias.bias_map(q, tol=1e-13)
    assert res.converged
    wn = p.wn * np.ones(p.N.shape)
    ref = np.vectorize(lambda N, w: bias.bias_closed_form_cell(N, w, p.mu, sigma2, b0))(p.N, wn)
    assert np.max(np.abs(res.s - ref) / np.maximum(np.abs(ref), 1.0)) <= 1e-10


def test_gradient_and_hessian_finite_differences():
    rng = np.random.default_rng(3)
    n, box = 8, 60.0
    p = _problem(n, box, rng, True, dc=0.2)
    kb, b = _bias_table(n, box, 1.1, slope=0.15)
    q = bias.BiasProblem(p, bias.bias_multipliers(n, box, kb, b, 1.05))
    s = 0.3 * rng.standard_normal(p.N.shape)
    assert np.all(bias.galaxy_density(s, q)[p.N > 0] > 0)
    d = rng.standard_normal(p.N.shape)
    h = 1e-6
    fd = (bias.bias_neg_log_posterior(s + h * d, q) - bias.bias_neg_log_posterior(s - h * d, q)) / (2 * h)
    an = float(np.sum(bias.bias_gradient(s, q) * d))
    assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0)
    v = rng.standard_normal(p.N.shape)
    fdh = (bias.bias_gradient(s + h * v, q) - bias.bias_gradient(s - h * v, q)) / (2 * h)
    hv = bias.bias_hessvec(s, v, q)
    assert np.max(np.abs(fdh - hv)) <= 1e-6 * np.max(np.abs(hv))


def test_hessian_is_symmetric():
    """B is symmetric (b depends on |k| only), so H = S^-1 + diag(e^s B q)
    + diag(e^s) B diag(N/u^2) B diag(e^s) is too."""
    rng = np.random.default_rng(11)
    n, box = 8, 60.0
    p = _problem(n, box, rng, True, dc=0.2)
    kb, b = _bias_table(n, box, 1.2, slope=-0.1)
    q = bias.BiasProblem(p, bias.bias_multipliers(n, box, kb, b, 1.2))
    s = 0.2 * rng.standard_normal(p.N.shape)
    u, v = rng.standard_normal(s.shape), rng.standard_normal(s.shape)
    a = float(np.sum(u * bias.bias_hessvec(s, v, q)))
    c = float(np.sum(v * bias.bias_hessvec(s, u, q)))
    assert abs(a - c) <= 1e-12 * max(abs(a), abs(c))
