"""GPU parity of the LSQ-Wiener filter (plc_wiener_lsq) against the oracle.

Bars: FP64 every element within 1e-10 of the solution's largest element,
and relative L2 <= 1e-10, of the oracle's solution (both to relative
residual 1e-12: the error is the residual times the inverse operator's
norm, a few hundred here); PLC_MIXED (FP32 CG) relative L2 <= 1e-5 and
every element within 5e-5 of the largest at residual 1e-6 (the same
argument at 1e-6 plus the FP32 rounding of the iterate).
At the full workload sizes the GPU solution's residual is taken with the
oracle's own FP64 operator.
"""
import math

import numpy as np
import pytest
import torch

from oracle import filters, plc as orc
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host, max_rel, rel_l2, small_mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _ctx(plc, m, precision):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    return c


def _problem(m):
    return orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)


@pytest.mark.parametrize("n,sel", [(24, "radial_masked"), (32, "uniform"), (48, "radial_masked"),
                                   (18, "uniform")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lsq_matches_oracle(plc, n, sel, precision):
    m = small_mock(n, sel, sigma=1.3, nbar=0.8)
    ref, cg = filters.wiener_lsq(_problem(m), rtol=1e-13)
    c = _ctx(plc, m, precision)
    tol = 1e-12 if precision == "fp64" else 1e-6
    d, st, stats = c.wiener_lsq(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=tol)
    assert st == 0 and stats["grad_rel"] <= tol
    assert rel_l2(host(d), ref) <= (1e-10 if precision == "fp64" else 1e-5)
    assert max_rel(host(d), ref) <= (1e-10 if precision == "fp64" else 5e-5)


def test_lsq_diagonal_prior_closed_form(plc):
    n, box, sigma2 = 16, 80.0, 0.9
    rng = np.random.default_rng(3)
    N = rng.poisson(2.0, size=(n, n, n)).astype(np.int32)
    w = rng.uniform(0.05, 1.0, size=(n, n, n))
    nbar = 1.6
    k = np.array([0.5 * 2 * math.pi / box, 2 * math.sqrt(3) * math.pi * n / box])
    P = np.full(2, sigma2 * box ** 3 / n ** 3)
    c = plc.Context(n, box, "fp64")
    c.set_prior(k, P, 0.0, 1.0 / sigma2)
    d, st, _ = c.wiener_lsq(dev(N, torch.int32), dev(w, torch.float64), nbar, tol=1e-13)
    exact = filters.wiener_closed_form_diagonal(N, w, nbar, sigma2)
    assert np.max(np.abs(host(d) - exact)) <= 1e-11 * np.max(np.abs(exact))


@pytest.mark.parametrize("key,precision", [("selection128", "fp64"), ("selection128", "mixed"),
                                           ("production256", "mixed")])
def test_lsq_full_size_residual_by_the_oracle(plc, key, precision):
    m = mocks.make_mock(mocks.WORKLOADS[key])
    c = _ctx(plc, m, precision)
    tol = 1e-10 if precision == "fp64" else 1e-6
    d, st, stats = c.wiener_lsq(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=tol)
    assert st == 0
    p = _problem(m)
    delta = host(d)
    wn = p.wn * np.ones(m.N.shape)
    b = m.N - wn
    res = orc.apply_Sinv(delta, p.inv_lam) + wn * delta - b
    # FP64: the CG's recursive residual and the true one agree to rounding;
    # FP32 CG: the true residual sits at the FP32 rounding level
    bar = 2.0 * tol if precision == "fp64" else 1e-5
    assert np.linalg.norm(res) / np.linalg.norm(b) <= bar


# ------------------------- Gaussian prior, Poisson likelihood ---------------

_GAUSS_CACHE = {}


def _gauss_ref(key, m, tol=1e-12):
    if key not in _GAUSS_CACHE:
        _GAUSS_CACHE[key] = filters.gauss_map(_problem(m), tol=tol)
    return _GAUSS_CACHE[key]


def _gauss_mock(key):
    if key == "g24":
        return small_mock(24, "radial_masked", sigma=1.2, nbar=1.0)
    if key == "g32":
        return small_mock(32, "uniform", sigma=1.0, nbar=2.0)
    raise KeyError(key)


@pytest.mark.parametrize("key", ["g24", "g32"])
def test_gauss_map_fp64_matches_oracle(plc, key):
    m = _gauss_mock(key)
    ref = _gauss_ref(key, m)
    assert ref.converged
    c = _ctx(plc, m, "fp64")
    r = c.gauss_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=1e-12)
    assert r.stats["grad_rel"] < 1e-12
    d = host(r.s)
    err = np.abs(d - ref.delta) / np.maximum(np.abs(ref.delta), 1.0)
    assert err.max() <= 1e-10
    assert np.all(1.0 + d[m.N > 0] > 0.0)


@pytest.mark.parametrize("key", ["g24", "g32"])
def test_gauss_map_mixed_matches_oracle(plc, key):
    m = _gauss_mock(key)
    ref = _gauss_ref(key, m)
    c = _ctx(plc, m, "mixed")
    r = c.gauss_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=1e-6)
    assert r.stats["grad_rel"] < 1e-6
    d = host(r.s)
    assert np.max(np.abs(d - ref.delta) / np.maximum(np.abs(ref.delta), 1.0)) <= 1e-4
    assert rel_l2(d, ref.delta) <= 1e-5


def test_gauss_map_diagonal_prior_closed_form(plc):
    n, box, sigma2 = 16, 80.0, 0.9
    rng = np.random.default_rng(13)
    N = rng.poisson(2.0, size=(n, n, n)).astype(np.int32)
    N[0, 0, 0] = 50
    w = rng.uniform(0.05, 1.0, size=(n, n, n))
    nbar = 1.6
    k = np.array([0.5 * 2 * math.pi / box, 2 * math.sqrt(3) * math.pi * n / box])
    P = np.full(2, sigma2 * box ** 3 / n ** 3)
    c = plc.Context(n, box, "fp64")
    c.set_prior(k, P, 0.0, 1.0 / sigma2)
    r = c.gauss_map(dev(N, torch.int32), dev(w, torch.float64), nbar, tol=1e-13)
    exact = filters.gauss_closed_form_diagonal(N, w, nbar, sigma2)
    err = np.abs(host(r.s) - exact) / np.maximum(np.abs(exact), 1.0)
    assert err.max() <= 1e-10


@pytest.mark.parametrize("key,precision", [("selection128", "fp64"), ("selection128", "mixed"),
                                           ("production256", "mixed")])
def test_gauss_map_full_size_is_a_map_for_the_oracle(plc, key, precision):
    m = mocks.make_mock(mocks.WORKLOADS[key])
    c = _ctx(plc, m, precision)
    r = c.gauss_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=1e-6)
    d = host(r.s)
    p = _problem(m)
    g0 = np.linalg.norm(filters.gauss_gradient(np.zeros(m.N.shape), p))
    rel = np.linalg.norm(filters.gauss_gradient(d, p)) / g0
    assert rel < 1e-6
    assert abs(rel - r.stats["grad_rel"]) <= 1e-3 * r.stats["grad_rel"]
    assert np.all(1.0 + d[m.N > 0] > 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gauss_map_start_option(plc, precision):
    """From delta = 0 (start = 0) or from the per-cell diagonal-prior MAP
    (start = 1): the same MAP, with ||g0|| taken at delta = 0 both times."""
    m = _gauss_mock("g32")
    ref = _gauss_ref("g32", m)
    c = _ctx(plc, m, precision)
    tol = 1e-12 if precision == "fp64" else 1e-6
    out = {}
    for start in (0, 1):
        r = c.gauss_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=tol,
                        start=start)
        assert r.stats["grad_rel"] < tol
        out[start] = (host(r.s), r.stats)
    # start = 1 takes ||g(0)|| = ||nbar w - N|| without a transform
    assert abs(out[0][1]["g0_norm"] - out[1][1]["g0_norm"]) <= 1e-6 * out[0][1]["g0_norm"]
    bar = 1e-10 if precision == "fp64" else 1e-4
    for start in (0, 1):
        d = out[start][0]
        assert np.max(np.abs(d - ref.delta) / np.maximum(np.abs(ref.delta), 1.0)) <= bar
