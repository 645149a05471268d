"""GPU parity of the operators against the FP64 oracle (through the C ABI).

Sizes span several tiles and a ragged tail: tiles are 8 (FP64) / 16 (FP32)
complex lines and 16 / 32 real rows, so n = 24, 48 and 96 leave partial
tiles along z, y and the n/2+1 kx lines; n = 4 and 6 are smaller than one
tile; n = 6, 18 and 54 (one factor of 2) take the one-element-per-step x
passes, the others the 4-wide ones; n = 32, 64, 96, 128, 192, 256 use the
four-step FP32 transforms.  FP64 bar: relative error <= 1e-12 (an FFT round trip
of length n^3 in double accumulates a few 1e-15 per stage).  FP32 bars
(PLC_MIXED operators), element by element and as a norm: every element
within 2e-5 of the reference's largest element, and relative L2 <= 1e-5.
Each output element is a sum over all n^3 inputs through ~log2(n^3) <= 27
butterfly stages per transform, two transforms, with rounding eps32 = 6e-8
per stage: ~2 x 27 x 6e-8 = 3.2e-6 of the transformed field's scale in the
worst case, times the spread of the multiplier 1/lambda across the modes
that carry the field (a few), plus the pointwise tail's rounding.
"""
import math

import numpy as np
import pytest
import torch

from oracle import plc as orc
from tests.gpu_util import dev, ensure_lib, host, max_rel, rel_l2, small_mock, pk_table_for

FP32_MAX = 2e-5     # element-wise bar of the FP32 operators (module docstring)

pytestmark = pytest.mark.gpu

SIZES = [4, 6, 8, 12, 18, 24, 48, 54, 96]


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _ctx(plc, n, box, precision, mu=-0.3, dc=0.0, seed=0):
    c = plc.Context(n, box, precision)
    k, P = pk_table_for(n, box, seed=seed)
    c.set_prior(k, P, mu, dc)
    inv = orc.inverse_eigenvalues(n, box, k, P, dc)
    return c, inv


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_prior_apply(plc, n, precision):
    box = 7.0 * n
    c, inv = _ctx(plc, n, box, precision, dc=0.37)
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n))
    ref = orc.apply_Sinv(x, inv)
    y = host(c.prior_apply(dev(x, c.real)))
    if precision == "fp64":
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    else:
        assert rel_l2(y, ref) <= 1e-5
        assert max_rel(y, ref) <= FP32_MAX


@pytest.mark.parametrize("n,mode", [(32, (0, 0, 1)), (32, (16, 3, 7)), (24, (12, 12, 12)),
                                    (48, (5, 20, 24))])
def test_single_mode_eigenvalue(plc, n, mode):
    box = 100.0
    c, inv = _ctx(plc, n, box, "fp64")
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    f = np.cos(2 * np.pi * (mode[0] * z + mode[1] * y + mode[2] * x) / n + 0.1)
    out = host(c.prior_apply(dev(f, torch.float64)))
    lam_inv = inv[mode]
    assert np.max(np.abs(out - lam_inv * f)) <= 1e-12 * lam_inv


@pytest.mark.parametrize("alpha1,alpha2", [(-1.7, 0.6), (1.0, -2.4)])
@pytest.mark.parametrize("n,mode_lo,mode_hi", [(12, (1, 2, 0), (3, 1, 4)), (24, (3, 2, 5), (9, 4, 7)),
                                               (32, (4, 1, 6), (13, 5, 9))])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_mode_between_table_nodes(plc, n, mode_lo, mode_hi, alpha1, alpha2, precision):
    """P(k) between table nodes (linear in (ln k, ln P)): a broken power law
    with its kink on a node makes the eigenvalue of an off-node mode exact,
    on both sides of the kink.  FP64 to 1e-12.  FP32 fields to 2e-5 of the
    peak element: the transforms' rounding (eps32 = 6e-8 times ~log2(n^3)
    = 15 stages) leaks into other modes, whose 1/lambda is up to ~10 times
    the mode's own for these tables."""
    from tests.test_oracle_operators import _kmag, broken_power_law_table
    box = 100.0
    k_lo, k_hi = _kmag(n, box, mode_lo), _kmag(n, box, mode_hi)
    k, P, P_lo, P_hi = broken_power_law_table(n, box, k_lo, k_hi, alpha1, alpha2)
    c = plc.Context(n, box, precision)
    c.set_prior(k, P, 0.0)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    for mode, Pq in ((mode_lo, P_lo), (mode_hi, P_hi)):
        f = np.cos(2 * np.pi * (mode[0] * z + mode[1] * y + mode[2] * x) / n - 0.7)
        ref = f * box ** 3 / (Pq * n ** 3)
        out = host(c.prior_apply(dev(f, c.real))).astype(np.float64)
        bar = 1e-12 if precision == "fp64" else 2e-5
        assert np.max(np.abs(out - ref)) <= bar * np.max(np.abs(ref))


@pytest.mark.parametrize("n,selection", [(8, "uniform"), (24, "radial_masked"), (48, "uniform")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_logpost_grad(plc, n, selection, precision):
    m = small_mock(n, selection)
    c = plc.Context(n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, n, m.box, m.k_tab, m.P_tab)
    rng = np.random.default_rng(3)
    s = m.mu + 0.7 * rng.standard_normal((n, n, n))
    f_ref = orc.neg_log_posterior(s, p)
    g_ref = orc.gradient(s, p)
    f, g = c.logpost_grad(dev(s, c.real), dev(m.N, torch.int32), dev(m.w, c.real), m.nbar)
    g = host(g)
    if precision == "fp64":
        assert abs(f - f_ref) <= 1e-12 * abs(f_ref)
        assert np.max(np.abs(g - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))
    else:
        # s itself is rounded to FP32: compare with the oracle at the rounded s
        s32 = s.astype(np.float32).astype(np.float64)
        assert abs(f - orc.neg_log_posterior(s32, p)) <= 1e-6 * abs(f_ref)
        g_ref32 = orc.gradient(s32, p)
        assert rel_l2(g, g_ref32) <= 1e-5
        assert max_rel(g, g_ref32) <= FP32_MAX


@pytest.mark.parametrize("n", [6, 24, 48, 96])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hessvec(plc, n, precision):
    m = small_mock(n, "radial_masked" if n >= 24 else "uniform")
    c = plc.Context(n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, n, m.box, m.k_tab, m.P_tab)
    rng = np.random.default_rng(4)
    s = m.mu + 0.7 * rng.standard_normal((n, n, n))
    v = rng.standard_normal((n, n, n))
    if precision == "mixed":
        s = s.astype(np.float32).astype(np.float64)
    ref = orc.hessvec(s, v, p)
    out = host(c.hessvec(dev(s, c.real), dev(m.w, c.real), m.nbar, dev(v, c.real)))
    if precision == "fp64":
        assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))
    else:
        assert rel_l2(out, ref) <= 1e-5
        assert max_rel(out, ref) <= FP32_MAX


def test_hessian_symmetric_and_pd_on_gpu(plc):
    n = 32
    m = small_mock(n)
    c = plc.Context(n, m.box, "fp64")
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    rng = np.random.default_rng(5)
    s = dev(m.mu + 0.5 * rng.standard_normal((n,) * 3), torch.float64)
    u = dev(rng.standard_normal((n,) * 3), torch.float64)
    v = dev(rng.standard_normal((n,) * 3), torch.float64)
    a = float((u * c.hessvec(s, None, m.nbar, v)).sum())
    b = float((v * c.hessvec(s, None, m.nbar, u)).sum())
    assert abs(a - b) <= 1e-12 * abs(a)
    assert float((v * c.hessvec(s, None, m.nbar, v)).sum()) > 0


def test_invalid_arguments(plc):
    with pytest.raises(plc.PlcError) as e:
        plc.Context(10, 100.0)          # prime factor 5
    assert e.value.status == 1
    with pytest.raises(plc.PlcError):
        plc.Context(7, 100.0)           # odd
    c = plc.Context(8, 100.0)
    x = c.field()
    with pytest.raises(plc.PlcError):
        c.prior_apply(x)                # no prior yet
    k = np.array([0.1, 0.2, 0.3])
    with pytest.raises(plc.PlcError):
        c.set_prior(k, np.ones(3), 0.0)  # does not cover the grid
    kk, P = pk_table_for(8, 100.0)
    with pytest.raises(plc.PlcError):
        c.set_prior(kk, -P, 0.0)         # negative power
    with pytest.raises(plc.PlcError):
        c.set_prior(kk[::-1].copy(), P, 0.0)   # not ascending
    c.set_prior(kk, P, 0.0)
    N = torch.zeros((8, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(plc.PlcError):
        c.logpost_grad(x, N, None, -1.0)       # nbar <= 0


_LARGE_REF = {}


def _large_case(n):
    """Oracle S^-1 x and H v at a production-sized grid (computed once)."""
    if n not in _LARGE_REF:
        box = 500.0 * n / 256
        k, P = pk_table_for(n, box, nbins=512, seed=1)
        inv = orc.inverse_eigenvalues(n, box, k, P, 0.0)
        rng = np.random.default_rng(100 + n)
        x = rng.standard_normal((n, n, n))
        s = -1.62 + 0.8 * rng.standard_normal((n, n, n))
        p = orc.Problem(np.zeros((n, n, n), np.int32), None, 1.0, -1.62, inv)
        # the mixed-precision operators see s rounded to FP32
        s32 = s.astype(np.float32).astype(np.float64)
        _LARGE_REF[n] = dict(box=box, k=k, P=P, x=x, s=s, s32=s32,
                             sinv=orc.apply_Sinv(x, inv),
                             hv64=orc.hessvec(s, x, p), hv32=orc.hessvec(s32, x, p))
    return _LARGE_REF[n]


@pytest.mark.parametrize("n", [128, 192, 256])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_operators_at_production_sizes(plc, n, precision):
    """Full-size grids, where the FP32 passes use the register-resident
    four-step transforms (16x8, 16x12, 16x16) and FP64 the Stockham stages."""
    r = _large_case(n)
    c = plc.Context(n, r["box"], precision)
    c.set_prior(r["k"], r["P"], -1.62)
    y = host(c.prior_apply(dev(r["x"], c.real)))
    s = r["s"] if precision == "fp64" else r["s32"]
    hv = host(c.hessvec(dev(s, c.real), None, 1.0, dev(r["x"], c.real)))
    if precision == "fp64":
        assert np.max(np.abs(y - r["sinv"])) <= 1e-12 * np.max(np.abs(r["sinv"]))
        assert np.max(np.abs(hv - r["hv64"])) <= 1e-12 * np.max(np.abs(r["hv64"]))
    else:
        assert rel_l2(y, r["sinv"]) <= 1e-5
        assert rel_l2(hv, r["hv32"]) <= 1e-5
        assert max_rel(y, r["sinv"]) <= FP32_MAX
        assert max_rel(hv, r["hv32"]) <= FP32_MAX
