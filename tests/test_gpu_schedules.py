"""Every FP32 line-transform schedule (register four-step n = f1 f2 in each
offered factor order, and the shared-memory Stockham stages) computes the
same operators, and the autotuner picks one of them.

The schedules offered per n are those of the library's table (ctx.h,
kFourStep); lengths without a four-step form (24, 48, 54: ragged tiles)
run the Stockham stages only.  FP32 bars as in test_gpu_operators: every
element within 2e-5 of the reference's largest, relative L2 <= 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import plc as orc
from tests.gpu_util import dev, ensure_lib, host, max_rel, rel_l2, pk_table_for

pytestmark = pytest.mark.gpu

OFFERED = {256: [(16, 16)], 192: [(16, 12), (12, 16)], 128: [(16, 8), (8, 16)],
           96: [(12, 8), (8, 12)], 64: [(8, 8)], 32: [(8, 4)], 24: [], 48: [], 54: []}


def _close(out, ref):
    return rel_l2(out, ref) <= 1e-5 and max_rel(out, ref) <= 2e-5


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


@pytest.mark.parametrize("n", [24, 32, 48, 54, 64, 96, 128, 192])
def test_every_schedule_matches_the_oracle(plc, n):
    box, mu, nbar = 6.0 * n, -0.4, 1.3
    k, P = pk_table_for(n, box, seed=n)
    c = plc.Context(n, box, "mixed")
    c.set_prior(k, P, mu)
    p_inv = orc.inverse_eigenvalues(n, box, k, P)
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n))
    s = (mu + 0.5 * rng.standard_normal((n, n, n))).astype(np.float32).astype(np.float64)
    v = rng.standard_normal((n, n, n)).astype(np.float32).astype(np.float64)
    N = rng.poisson(1.5, size=(n, n, n)).astype(np.int32)
    prob = orc.Problem(N, None, nbar, mu, p_inv)
    ref_y = orc.apply_Sinv(x, p_inv)
    ref_hv = orc.hessvec(s, v, prob)
    ref_g = orc.gradient(s, prob)
    xs, ss, vs, Nd = dev(x, torch.float32), dev(s, torch.float32), dev(v, torch.float32), dev(N, torch.int32)
    for f1, f2 in [(0, 0)] + OFFERED[n]:
        c.set_fft_schedule(f1, f2)
        assert _close(host(c.prior_apply(xs)), ref_y), (f1, f2)
        assert _close(host(c.hessvec(ss, None, nbar, vs)), ref_hv), (f1, f2)
        _, g = c.logpost_grad(ss, Nd, None, nbar)
        assert _close(host(g), ref_g), (f1, f2)
    f1, f2, us = c.autotune(reps=5)
    assert (f1, f2) in [(0, 0)] + OFFERED[n] and us > 0.0
    assert _close(host(c.prior_apply(xs)), ref_y)


def test_schedule_validation(plc):
    c = plc.Context(64, 300.0, "mixed")
    with pytest.raises(plc.PlcError):
        c.set_fft_schedule(16, 4)      # not offered for 64
    with pytest.raises(plc.PlcError):
        c.set_fft_schedule(8, 16)      # product is not n
    c.set_fft_schedule(0, 0)
    c64 = plc.Context(64, 300.0, "fp64")
    k, P = pk_table_for(64, 300.0)
    c64.set_prior(k, P, -0.3)
    assert c64.autotune(reps=2)[2] == 0.0   # FP64 transforms have one schedule


def test_autotuned_map_equals_default_within_tolerance(plc):
    """A MAP solved with the autotuned schedule is a MAP (same stop test) and
    agrees with the default schedule's to the mixed-precision bar."""
    from paper_0911_1407_gb300 import mocks
    m = mocks.make_mock(mocks.WORKLOADS["adjoint128"])
    c = plc.Context(m.n, m.box, "mixed")
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    Nd = dev(m.N, torch.int32)
    r0 = c.newton_krylov_map(Nd, None, m.nbar)
    c.set_fft_schedule(8, 16)
    r1 = c.newton_krylov_map(Nd, None, m.nbar)
    assert r0.stats["grad_rel"] < 1e-6 and r1.stats["grad_rel"] < 1e-6
    d = host(r0.s) - host(r1.s)
    assert np.max(np.abs(d)) <= 1e-4
