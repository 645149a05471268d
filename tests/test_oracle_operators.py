"""Pins for the oracle's prior operator, objective, gradient and Hessian.

* S^-1 on a single Fourier mode is a scalar multiple 1/lambda_k (Sec. 2.2),
  with lambda_k = P(|k|) n^3 / L^3 read straight off a table node.
* Between table nodes P is linear in (ln k, ln P), which is exact for a
  power law: a broken power law with its kink on a node gives the
  eigenvalue of an off-node mode in closed form, on either side of the kink.
* The gradient (Sec. 3.1.2) is the derivative of the objective (prior of
  Sec. 2.3 plus likelihood of Sec. 2.1): central finite differences.
* The Hessian (Sec. 3.1.2) is the derivative of the gradient, symmetric and
  positive definite.
"""
import math

import numpy as np
import pytest

from oracle import plc


def _table_with_node(n, box, kq, Pq, nbins=64):
    """A P(k) table covering the grid that has (kq, Pq) as an exact node."""
    kf = 2 * math.pi / box
    kmax = 1.01 * math.sqrt(3) * math.pi * n / box
    k = np.unique(np.concatenate([np.exp(np.linspace(math.log(0.5 * kf), math.log(kmax), nbins)), [kq]]))
    P = 100.0 * (1 + 0.3 * np.sin(5 * np.log(k)))   # smooth, positive, not a power law
    P[k == kq] = Pq
    return k, P


@pytest.mark.parametrize("n,mode", [(8, (0, 0, 1)), (8, (2, 3, 1)), (8, (4, 0, 0)),
                                    (12, (5, 6, 3)), (6, (3, 3, 3))])
def test_single_mode_eigenvalue(n, mode):
    box = 100.0
    mz, my, mx = mode
    msigned = [m if m <= n // 2 else m - n for m in mode]
    kq = 2 * math.pi / box * math.sqrt(sum(m * m for m in msigned))
    Pq = 37.5
    k_tab, P_tab = _table_with_node(n, box, kq, Pq)
    inv = plc.inverse_eigenvalues(n, box, k_tab, P_tab)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    field = np.cos(2 * np.pi * (mz * z + my * y + mx * x) / n + 0.3)
    lam = Pq * n ** 3 / box ** 3
    out = plc.apply_Sinv(field, inv)
    assert np.max(np.abs(out - field / lam)) < 1e-12 * np.max(np.abs(field / lam))


def broken_power_law_table(n, box, k_lo, k_hi, alpha1, alpha2, A=50.0):
    """Table of P = A (k/k_b)^alpha1 below k_b and A (k/k_b)^alpha2 above it,
    k_b = sqrt(k_lo k_hi), on log nodes k_b e^{j h} with h = 0.8 ln(k_hi/k_lo):
    k_lo and k_hi then sit strictly inside the two segments next to the kink,
    at fractions 0.375 and 0.625 of a segment.  Returns the table and the
    exact P at k_lo and k_hi."""
    kb = math.sqrt(k_lo * k_hi)
    h = 0.8 * math.log(k_hi / k_lo)
    kmin, kmax = 0.5 * 2 * math.pi / box, 1.01 * math.sqrt(3) * math.pi * n / box
    j = np.arange(math.floor(math.log(kmin / kb) / h), math.ceil(math.log(kmax / kb) / h) + 1)
    k = kb * np.exp(h * j)

    def P(x):
        return A * (x / kb) ** np.where(x < kb, alpha1, alpha2)
    return k, P(k), float(P(np.array(k_lo))), float(P(np.array(k_hi)))


def _kmag(n, box, mode):
    ms = [m if m <= n // 2 else m - n for m in mode]
    return 2 * math.pi / box * math.sqrt(sum(m * m for m in ms))


@pytest.mark.parametrize("alpha1,alpha2", [(-1.7, 0.6), (1.0, -2.4), (0.5, 0.5)])
@pytest.mark.parametrize("n,mode_lo,mode_hi", [(8, (0, 1, 1), (2, 1, 2)), (12, (1, 2, 0), (3, 1, 4)),
                                               (16, (2, 3, 5), (7, 1, 6))])
def test_single_mode_between_table_nodes(n, mode_lo, mode_hi, alpha1, alpha2):
    box = 100.0
    k_lo, k_hi = _kmag(n, box, mode_lo), _kmag(n, box, mode_hi)
    k_tab, P_tab, P_lo, P_hi = broken_power_law_table(n, box, k_lo, k_hi, alpha1, alpha2)
    # both modes lie strictly between nodes (at least 1/4 of a segment away)
    lk = np.log(k_tab)
    for kq in (k_lo, k_hi):
        gap = np.min(np.abs(lk - math.log(kq))) / (lk[1] - lk[0])
        assert gap > 0.25
    inv = plc.inverse_eigenvalues(n, box, k_tab, P_tab)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    for mode, Pq in ((mode_lo, P_lo), (mode_hi, P_hi)):
        f = np.cos(2 * np.pi * (mode[0] * z + mode[1] * y + mode[2] * x) / n - 0.7)
        ref = f * box ** 3 / (Pq * n ** 3)
        out = plc.apply_Sinv(f, inv)
        assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dc_rule():
    n, box = 8, 50.0
    k_tab, P_tab = _table_with_node(n, box, 0.5, 1.0)
    const = np.full((n, n, n), 3.0)
    assert np.max(np.abs(plc.apply_Sinv(const, plc.inverse_eigenvalues(n, box, k_tab, P_tab)))) < 1e-13
    inv = plc.inverse_eigenvalues(n, box, k_tab, P_tab, inv_lambda_dc=0.25)
    assert np.allclose(plc.apply_Sinv(const, inv), 0.75, rtol=1e-13, atol=0)


def test_table_coverage_is_checked():
    n, box = 8, 50.0
    k = np.array([0.2, 0.3, 0.4])
    with pytest.raises(ValueError):
        plc.inverse_eigenvalues(n, box, k, np.ones(3))


def _problem(n=8, seed=5, with_w=True):
    rng = np.random.default_rng(seed)
    box = 80.0
    kf = 2 * math.pi / box
    k = np.exp(np.linspace(math.log(0.5 * kf), math.log(1.01 * math.sqrt(3) * math.pi * n / box), 40))
    P = 200.0 * k / (1 + (k / 0.05) ** 2) ** 1.4
    N = rng.poisson(2.0, size=(n, n, n))
    w = rng.uniform(0.2, 1.0, size=(n, n, n)) if with_w else None
    p = plc.make_problem(N, w, 1.7, -0.4, n, box, k, P)
    s = -0.4 + 0.5 * rng.standard_normal((n, n, n))
    return p, s, rng


@pytest.mark.parametrize("with_w", [True, False])
def test_gradient_matches_finite_differences(with_w):
    p, s, rng = _problem(with_w=with_w)
    g = plc.gradient(s, p)
    for _ in range(3):
        u = rng.standard_normal(s.shape)
        eps = 1e-6
        fd = (plc.neg_log_posterior(s + eps * u, p) - plc.neg_log_posterior(s - eps * u, p)) / (2 * eps)
        assert abs(fd - np.sum(u * g)) <= 1e-7 * abs(fd) + 1e-9


def test_hessvec_matches_finite_differences_of_gradient():
    p, s, rng = _problem()
    v = rng.standard_normal(s.shape)
    eps = 1e-6
    fd = (plc.gradient(s + eps * v, p) - plc.gradient(s - eps * v, p)) / (2 * eps)
    hv = plc.hessvec(s, v, p)
    assert np.linalg.norm(fd - hv) <= 1e-7 * np.linalg.norm(hv)


def test_hessian_symmetric_positive_definite():
    p, s, rng = _problem()
    u, v = rng.standard_normal(s.shape), rng.standard_normal(s.shape)
    a = np.sum(u * plc.hessvec(s, v, p))
    b = np.sum(v * plc.hessvec(s, u, p))
    assert abs(a - b) <= 1e-13 * max(abs(a), abs(b))
    for _ in range(5):
        x = rng.standard_normal(s.shape)
        assert np.sum(x * plc.hessvec(s, x, p)) > 0


def test_gradient_vanishes_term_by_term_structure():
    """With the prior switched off (1/lambda = 0) the gradient is D - N."""
    p, s, _ = _problem()
    p0 = plc.Problem(p.N, p.w, p.nbar, p.mu, np.zeros_like(p.inv_lam))
    assert np.allclose(plc.gradient(s, p0), p.nbar * p.w * np.exp(s) - p.N, rtol=1e-14, atol=1e-12)
