"""GPU parity of the Newton-Krylov MAP and its adjoint against the oracle.

Bars: FP64 GPU MAP within a per-voxel relative error of 1e-10
(|s - s_ref| / max(|s_ref|, 1)) of the oracle, both converged to
||g|| / ||g0|| < 1e-12.  Mixed precision stopped at 1e-6: max-abs error
<= 1e-4 and relative-L2 <= 1e-5 against the FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

from oracle import plc as orc
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host, max_rel, rel_l2, small_mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


_ORACLE_CACHE = {}


def _oracle_map(key, m, tol=1e-12):
    if key not in _ORACLE_CACHE:
        p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
        _ORACLE_CACHE[key] = (p, orc.newton_krylov_map(p, tol=tol))
    return _ORACLE_CACHE[key]


def _mock(key):
    if key == "plain32":
        return mocks.make_mock(mocks.WORKLOADS["plain32"])
    if key == "sel24":
        return small_mock(24, "radial_masked", sigma=1.3, nbar=1.0)
    if key == "sel48":
        return small_mock(48, "radial_masked", sigma=1.5, nbar=0.5)
    raise KeyError(key)


def _gpu_map(plc, m, precision, tol, **kw):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    r = c.newton_krylov_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, tol=tol, **kw)
    return host(r.s), r.stats


@pytest.mark.parametrize("key", ["plain32", "sel24", "sel48"])
def test_map_fp64_matches_oracle(plc, key):
    m = _mock(key)
    p, ref = _oracle_map(key, m)
    assert ref.converged
    s, st = _gpu_map(plc, m, "fp64", 1e-12)
    assert st["grad_rel"] < 1e-12
    err = np.abs(s - ref.s) / np.maximum(np.abs(ref.s), 1.0)
    assert err.max() <= 1e-10
    # DC of the gradient vanishes at the MAP: sum w nbar e^s = sum N
    D = p.wn * np.exp(s)
    assert abs(D.sum() - m.N.sum()) <= 1e-9 * m.N.sum()


@pytest.mark.parametrize("key", ["plain32", "sel24", "sel48"])
def test_map_mixed_matches_oracle(plc, key):
    m = _mock(key)
    _, ref = _oracle_map(key, m)
    s, st = _gpu_map(plc, m, "mixed", 1e-6)
    assert st["grad_rel"] < 1e-6
    assert np.max(np.abs(s - ref.s)) <= 1e-4
    assert rel_l2(s, ref.s) <= 1e-5


def test_map_diagonal_prior_closed_form(plc):
    n, box, sigma2 = 16, 80.0, 0.9
    rng = np.random.default_rng(7)
    N = rng.poisson(2.5, size=(n, n, n)).astype(np.int32)
    N[0, 0, 0] = 60
    w = rng.uniform(0.05, 1.0, size=(n, n, n))
    nbar, mu = 1.4, -0.45
    k = np.array([0.5 * 2 * math.pi / box, 2 * math.sqrt(3) * math.pi * n / box])
    P = np.full(2, sigma2 * box ** 3 / n ** 3)
    c = plc.Context(n, box, "fp64")
    c.set_prior(k, P, mu, 1.0 / sigma2)
    r = c.newton_krylov_map(dev(N, torch.int32), dev(w, torch.float64), nbar, tol=1e-13)
    exact = orc.map_closed_form_diagonal(N, w, nbar, mu, sigma2)
    err = np.abs(host(r.s) - exact) / np.maximum(np.abs(exact), 1.0)
    assert err.max() <= 1e-10


def test_map_resume_and_cap(plc):
    m = _mock("plain32")
    c = plc.Context(m.n, m.box, "fp64")
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    Nd = dev(m.N, torch.int32)
    r1 = c.newton_krylov_map(Nd, None, m.nbar, tol=1e-12, max_newton=2, raise_on_fail=False)
    assert r1.status == 3 and r1.stats["newton_iters"] == 2
    # resume from the last iterate with the original ||g0||
    r2 = c.newton_krylov_map(Nd, None, m.nbar, s=r1.s, tol=1e-12, g0_norm=r1.stats["g0_norm"])
    _, ref = _oracle_map("plain32", m)
    assert np.max(np.abs(host(r2.s) - ref.s) / np.maximum(np.abs(ref.s), 1)) <= 1e-10


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_vjp_matches_oracle(plc, precision, bar):
    m = small_mock(16, "uniform", sigma=1.0, nbar=2.0)
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    ref = orc.newton_krylov_map(p, tol=1e-13)
    u = np.random.default_rng(2).standard_normal(m.N.shape)
    lam_ref, lnA_ref, _ = orc.map_vjp(ref.s, u, p, rtol=1e-13)
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    tol = 1e-13 if precision == "fp64" else 1e-6
    vN, vA, st = c.map_vjp(dev(ref.s, torch.float64), None, m.nbar, dev(u, torch.float64), tol=tol)
    assert rel_l2(host(vN), lam_ref) <= bar
    assert max_rel(host(vN), lam_ref) <= bar
    assert abs(vA - lnA_ref) <= bar * abs(lnA_ref)


@pytest.mark.parametrize("key,precision", [("selection128", "fp64"), ("selection128", "mixed"),
                                           ("production256", "mixed")])
def test_map_full_size_is_a_map_for_the_oracle(plc, key, precision):
    """At the full workload sizes the GPU MAP (stopped at ||g|| / ||g0|| < 1e-6)
    must be a MAP by the oracle's own gradient: one FP64 oracle gradient at
    s_gpu gives the same relative norm, below the tolerance, and the flat-mean
    invariant sum w nbar e^s = sum N holds."""
    m = mocks.make_mock(mocks.WORKLOADS[key])
    s, st = _gpu_map(plc, m, precision, 1e-6)
    assert st["grad_rel"] < 1e-6
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    g0 = np.linalg.norm(orc.gradient(np.full(m.N.shape, m.mu), p))
    rel = np.linalg.norm(orc.gradient(s, p)) / g0
    assert rel < 1e-6
    assert abs(rel - st["grad_rel"]) <= 1e-3 * st["grad_rel"]
    D = p.wn * np.exp(s)
    assert abs(D.sum() - m.N.sum()) <= 1e-4 * m.N.sum()


def test_map_mixed_vs_fp64_selection128(plc):
    """128^3 with radial selection and angular mask: the mixed-precision MAP
    against the FP64 GPU MAP, both stopped at ||g|| / ||g0|| < 1e-6."""
    m = mocks.make_mock(mocks.WORKLOADS["selection128"])
    s64, _ = _gpu_map(plc, m, "fp64", 1e-6)
    s32, _ = _gpu_map(plc, m, "mixed", 1e-6)
    assert np.max(np.abs(s32 - s64)) <= 1e-4
    assert rel_l2(s32, s64) <= 1e-5


@pytest.mark.parametrize("key", ["plain32", "sel48"])
def test_map_mixed_to_fp64_accuracy(plc, key):
    """The mixed form driven to ||g|| / ||g0|| < 1e-10: past the switch the
    state, gradient and stop test are FP64 (the refresh gradient through
    float-float transforms at 32^3, FP64 Stockham at 48^3) while the CG stays
    FP32, so the iteration refines to the FP64 MAP (per-voxel 1e-8)."""
    m = _mock(key)
    _, ref = _oracle_map(key, m)
    s, st = _gpu_map(plc, m, "mixed", 1e-10)
    assert st["grad_rel"] < 1e-10 and st["grad_ffts_fp64"] >= 1
    err = np.abs(s - ref.s) / np.maximum(np.abs(ref.s), 1.0)
    assert err.max() <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_map_start_point_option(plc, precision):
    """The diagonal-prior start (opts.start = 1) reaches the same MAP as the
    start at mu with fewer Newton steps; ||g0|| is taken at mu in both (with
    start = 1 by the transform-free form g(mu) = nbar w e^mu - N, summed in
    compensated FP32, so equal to ~1e-7)."""
    m = mocks.make_mock(mocks.WORKLOADS["adjoint128"])
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    Nd = dev(m.N, torch.int32)
    tol = 1e-10 if precision == "fp64" else 1e-6
    r0 = c.newton_krylov_map(Nd, None, m.nbar, tol=tol, start=0)
    r1 = c.newton_krylov_map(Nd, None, m.nbar, tol=tol, start=1)
    assert abs(r0.stats["g0_norm"] - r1.stats["g0_norm"]) <= 1e-6 * r0.stats["g0_norm"]
    assert r1.stats["newton_iters"] < r0.stats["newton_iters"]
    assert r1.stats["grad_ffts"] == r0.stats["grad_ffts"]      # no transform for g(mu)
    bar = 1e-8 if precision == "fp64" else 1e-4
    assert np.max(np.abs(host(r0.s) - host(r1.s))) <= bar


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("driven", [0, 1])
def test_start_at_mean_reads_no_start_array(plc, precision, driven):
    """opts.start = 2 is opts.start = 1 with the caller's start taken to be
    mu without reading the array: on an array full of NaN it gives the same
    MAP, bit for bit, and the same statistics as start = 1 on an array
    filled with mu (selection and angular mask, so w is read)."""
    m = _mock("sel24")
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    Nd, wd = dev(m.N, torch.int32), dev(m.w, torch.float64)
    tol = 1e-10 if precision == "fp64" else 1e-6
    s1 = torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda")
    s2 = torch.full((m.n,) * 3, float("nan"), dtype=torch.float64, device="cuda")
    r1 = c.newton_krylov_map(Nd, wd, m.nbar, s=s1, tol=tol, start=1, device_driven=driven)
    r2 = c.newton_krylov_map(Nd, wd, m.nbar, s=s2, tol=tol, start=2, device_driven=driven)
    assert torch.equal(s1, s2)
    for k in ("newton_iters", "cg_iters", "grad_evals", "grad_ffts", "grad_ffts_fp64",
              "g0_norm", "grad_rel", "neg_logpost"):
        assert r1.stats[k] == r2.stats[k], k
    if driven:
        # the same kernels less the control kernel of the never-taken IF node
        # that start = 1 keeps for a start off the mean
        assert r2.stats["kernels"] == r1.stats["kernels"] - 1


def test_gauss_map_start_at_zero_reads_no_start_array(plc):
    """The same option for the Gaussian-prior model: delta taken to be 0."""
    m = _mock("sel24")
    c = plc.Context(m.n, m.box, "fp64")
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    Nd, wd = dev(m.N, torch.int32), dev(m.w, torch.float64)
    d1 = torch.zeros((m.n,) * 3, dtype=torch.float64, device="cuda")
    d2 = torch.full((m.n,) * 3, float("nan"), dtype=torch.float64, device="cuda")
    r1 = c.gauss_map(Nd, wd, m.nbar, delta=d1, tol=1e-10, start=1)
    r2 = c.gauss_map(Nd, wd, m.nbar, delta=d2, tol=1e-10, start=2)
    assert torch.equal(d1, d2)
    for k in ("newton_iters", "cg_iters", "grad_evals", "g0_norm", "grad_rel"):
        assert r1.stats[k] == r2.stats[k], k
