"""GPU parity of the linear-bias model (Sec. 2.4.1) against the oracle.

* -ln P, gradient and exact Hessian-vector product element by element
  (FP64: 1e-11 relative to the field's scale; FP32 fields of PLC_MIXED:
  2e-4 of the field's scale, the FP32 rounding of three transforms).
* b = 1: the bias operators equal the unity-bias ones, and the bias MAP the
  unity-bias MAP.
* MAP parity with scale-dependent bias tables (FP64 per voxel 1e-9 of
  max(|s|, 1); PLC_MIXED to ||g||/||g0|| < 1e-6: 1e-4 per voxel).
* Constant bias and diagonal prior: per-cell bisection (brute force).
* production256 with the bias table: the oracle's own gradient at the GPU
  MAP.
"""
import math

import numpy as np
import pytest
import torch

from oracle import bias as ob, plc as orc
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host, rel_l2, small_mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _problem(m):
    return orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)


def _ctx(plc, m, precision, kb, b, b_dc):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    c.set_bias(kb, b, b_dc)
    return c


def _bp(m, kb, b, b_dc):
    return ob.BiasProblem(_problem(m), ob.bias_multipliers(m.n, m.box, kb, b, b_dc))


def _point(m, seed, amp=0.1):
    """A point inside the domain u > 0 for the tables used here (white noise
    of small amplitude around delta_M = 0)."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((m.n,) * 3)


@pytest.mark.parametrize("n,sel,b0,tilt", [(24, "radial_masked", 1.4, 0.1), (18, "uniform", 0.8, -0.2),
                                           (32, "uniform", 1.6, 0.15)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_operators_match_oracle(plc, n, sel, b0, tilt, precision):
    m = small_mock(n, sel, sigma=1.0, nbar=1.5)
    kb, b = mocks.bias_table(m.n, m.box, b0, tilt)
    q = _bp(m, kb, b, b0)
    s = _point(m, n)
    v = np.random.default_rng(n + 1).standard_normal(s.shape)
    f_ref = ob.bias_neg_log_posterior(s, q)
    assert math.isfinite(f_ref)
    g_ref = ob.bias_gradient(s, q)
    h_ref = ob.bias_hessvec(s, v, q)
    c = _ctx(plc, m, precision, kb, b, b0)
    real = torch.float64 if precision == "fp64" else torch.float32
    N, w = dev(m.N, torch.int32), dev(m.w, torch.float64)
    f, g = c.bias_logpost_grad(dev(s, real), N, w, m.nbar)
    hv = c.bias_hessvec(dev(s, real), N, w, m.nbar, dev(v, real))
    bar = 1e-11 if precision == "fp64" else 2e-4
    assert abs(f - f_ref) <= bar * max(abs(f_ref), 1.0) * (1 if precision == "fp64" else 10)
    assert np.max(np.abs(host(g) - g_ref)) <= bar * np.max(np.abs(g_ref))
    assert np.max(np.abs(host(hv) - h_ref)) <= bar * np.max(np.abs(h_ref))


def test_unit_bias_operators_equal_the_unity_bias_ones(plc):
    m = small_mock(24, "radial_masked", sigma=1.0, nbar=1.5)
    kb, b = mocks.bias_table(m.n, m.box, 1.0, 0.0)
    c = _ctx(plc, m, "fp64", kb, b, 1.0)
    s = dev(_point(m, 5), torch.float64)
    v = dev(np.random.default_rng(6).standard_normal((m.n,) * 3), torch.float64)
    N, w = dev(m.N, torch.int32), dev(m.w, torch.float64)
    fb, gb = c.bias_logpost_grad(s, N, w, m.nbar)
    fu, gu = c.logpost_grad(s, N, w, m.nbar)
    hb = c.bias_hessvec(s, N, w, m.nbar, v)
    hu = c.hessvec(s, w, m.nbar, v)
    # with b = 1, u = 1 + (e^s - 1) = e^s: the two models agree term by term
    assert abs(fb - fu) <= 1e-11 * abs(fu)
    assert rel_l2(host(gb), host(gu)) <= 1e-12
    assert rel_l2(host(hb), host(hu)) <= 1e-12


_MAP_CACHE = {}


def _map_case(key):
    if key == "b24":
        m = small_mock(24, "radial_masked", sigma=1.2, nbar=1.0)
        kb, b = mocks.bias_table(m.n, m.box, 1.5, 0.1)
        b_dc = 1.5
    elif key == "b32":
        m = small_mock(32, "uniform", sigma=1.0, nbar=2.0)
        kb, b = mocks.bias_table(m.n, m.box, 0.7, -0.15)
        b_dc = 0.9
    elif key == "unit24":
        m = small_mock(24, "radial_masked", sigma=1.2, nbar=1.0)
        kb, b = mocks.bias_table(m.n, m.box, 1.0, 0.0)
        b_dc = 1.0
    else:
        raise KeyError(key)
    if key not in _MAP_CACHE:
        _MAP_CACHE[key] = ob.bias_map(_bp(m, kb, b, b_dc), tol=1e-12)
    return m, kb, b, b_dc, _MAP_CACHE[key]


@pytest.mark.parametrize("key", ["b24", "b32", "unit24"])
def test_bias_map_fp64_matches_oracle(plc, key):
    m, kb, b, b_dc, ref = _map_case(key)
    assert ref.converged
    c = _ctx(plc, m, "fp64", kb, b, b_dc)
    r = c.bias_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=1e-12)
    assert r.stats["grad_rel"] < 1e-12
    s = host(r.s)
    assert np.max(np.abs(s - ref.s) / np.maximum(np.abs(ref.s), 1.0)) <= 1e-9
    assert abs(r.stats["neg_logpost"] - ref.neg_logpost) <= 1e-9 * abs(ref.neg_logpost)


@pytest.mark.parametrize("key", ["b24", "b32"])
def test_bias_map_mixed_matches_oracle(plc, key):
    m, kb, b, b_dc, ref = _map_case(key)
    c = _ctx(plc, m, "mixed", kb, b, b_dc)
    r = c.bias_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=1e-6)
    assert r.stats["grad_rel"] < 1e-6
    s = host(r.s)
    assert np.max(np.abs(s - ref.s) / np.maximum(np.abs(ref.s), 1.0)) <= 1e-4
    assert rel_l2(s, ref.s) <= 1e-5


def test_unit_bias_map_equals_unity_bias_map(plc):
    m, kb, b, b_dc, ref = _map_case("unit24")
    c = _ctx(plc, m, "fp64", kb, b, b_dc)
    N, w = dev(m.N, torch.int32), dev(m.w, torch.float64)
    rb = c.bias_map(N, w, m.nbar, tol=1e-12)
    ru = c.newton_krylov_map(N, w, m.nbar, tol=1e-12, device_driven=0)
    sb, su = host(rb.s), host(ru.s)
    assert np.max(np.abs(sb - su) / np.maximum(np.abs(su), 1.0)) <= 1e-9


@pytest.mark.parametrize("b0,sigma2", [(0.8, 1.2), (1.3, 0.7)])
def test_constant_bias_diagonal_prior_by_bisection(plc, b0, sigma2):
    n, box, nbar, mu = 16, 80.0, 1.3, -0.4
    rng = np.random.default_rng(int(b0 * 10) + 7)
    N = rng.poisson(2.0, size=(n, n, n)).astype(np.int32)
    N.flat[5] = 25
    w = rng.uniform(0.2, 1.0, size=(n, n, n))
    kf = 2 * math.pi / box
    k = np.array([0.5 * kf, 2 * math.sqrt(3) * math.pi * n / box])
    P = np.full(2, sigma2 * box ** 3 / n ** 3)
    c = plc.Context(n, box, "fp64")
    c.set_prior(k, P, mu, 1.0 / sigma2)
    c.set_bias(k, np.full(2, b0), b0)
    r = c.bias_map(dev(N, torch.int32), dev(w, torch.float64), nbar, tol=1e-13)
    ref = np.vectorize(lambda Ni, wi: ob.bias_closed_form_cell(Ni, wi, mu, sigma2, b0))(N, nbar * w)
    assert np.max(np.abs(host(r.s) - ref) / np.maximum(np.abs(ref), 1.0)) <= 1e-10


def test_bias_production256_is_a_map_for_the_oracle(plc):
    m = mocks.make_mock(mocks.WORKLOADS["production256"])
    kb, b = mocks.bias_table(m.n, m.box, 1.5, 0.1)
    c = _ctx(plc, m, "mixed", kb, b, 1.5)
    r = c.bias_map(dev(m.N, torch.int32), None, m.nbar, tol=1e-6)
    s = host(r.s)
    q = _bp(m, kb, b, 1.5)
    g0 = np.linalg.norm(ob.bias_gradient(np.zeros(s.shape), q))
    rel = np.linalg.norm(ob.bias_gradient(s, q)) / g0
    assert rel < 1e-6
    assert abs(rel - r.stats["grad_rel"]) <= 1e-3 * r.stats["grad_rel"] + 1e-9
    assert math.isfinite(ob.bias_neg_log_posterior(s, q))


def test_outside_the_domain_is_reported_as_non_finite(plc):
    m = small_mock(24, "radial_masked", sigma=1.0, nbar=1.5)
    kb, b = mocks.bias_table(m.n, m.box, 1.4, 0.1)
    s = m.mu + 0.3 * np.random.default_rng(24).standard_normal((m.n,) * 3)
    assert ob.bias_neg_log_posterior(s, _bp(m, kb, b, 1.4)) == math.inf
    c = _ctx(plc, m, "fp64", kb, b, 1.4)
    with pytest.raises(plc.PlcError) as e:
        c.bias_logpost_grad(dev(s, torch.float64), dev(m.N, torch.int32), dev(m.w, torch.float64),
                            m.nbar)
    assert e.value.status == 4


def test_bias_map_rejects_a_start_outside_the_domain(plc):
    m = small_mock(16, "uniform", sigma=1.0, nbar=2.0)
    kb, b = mocks.bias_table(m.n, m.box, 2.0, 0.0)
    c = _ctx(plc, m, "fp64", kb, b, 2.0)
    s = torch.full((m.n,) * 3, -5.0, dtype=torch.float64, device="cuda")   # u = 1 + 2 (e^-5 - 1) < 0
    r = c.bias_map(dev(m.N, torch.int32), None, m.nbar, s=s, raise_on_fail=False)
    assert r.status == 4      # PLC_ERR_NONFINITE
