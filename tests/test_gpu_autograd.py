"""torch.autograd front ends: backward passes against the oracle and finite
differences (the differentiation workload: sigma_G = 1.2, nbar = 1, w = 1)."""
import numpy as np
import pytest
import torch

from oracle import plc as orc
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host, max_rel, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _ctx(plc, m, precision):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    return c


def _start(m, seed=5):
    return m.mu + 0.4 * np.random.default_rng(seed).standard_normal(m.N.shape)


def test_neg_log_posterior_fp64_matches_oracle(plc):
    from paper_0911_1407_gb300.autograd import neg_log_posterior
    m = mocks.make_mock(mocks.WORKLOADS["adjoint32"])
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    s0 = _start(m)
    c = _ctx(plc, m, "fp64")
    s = dev(s0, torch.float64).requires_grad_(True)
    f = neg_log_posterior(s, c, dev(m.N, torch.int32), None, m.nbar)
    f.backward()
    f_ref = orc.neg_log_posterior(s0, p)
    assert abs(f.item() - f_ref) <= 1e-12 * abs(f_ref)
    assert rel_l2(host(s.grad), orc.gradient(s0, p)) <= 1e-12
    assert max_rel(host(s.grad), orc.gradient(s0, p)) <= 1e-12
    # the scale of grad_out passes through
    s.grad = None
    (3.0 * neg_log_posterior(s, c, dev(m.N, torch.int32), None, m.nbar)).backward()
    assert rel_l2(host(s.grad), 3.0 * orc.gradient(s0, p)) <= 1e-12


def test_neg_log_posterior_fp32_backward(plc):
    """FP32 backward at 128^3 against the FP64 gradient and a central
    difference of the FP64 objective along a random direction."""
    from paper_0911_1407_gb300.autograd import neg_log_posterior
    m = mocks.make_mock(mocks.WORKLOADS["adjoint128"])
    s0 = _start(m)
    Nd = dev(m.N, torch.int32)
    c32, c64 = _ctx(plc, m, "mixed"), _ctx(plc, m, "fp64")
    s32 = dev(s0, torch.float32).requires_grad_(True)
    neg_log_posterior(s32, c32, Nd, None, m.nbar).backward()
    s64 = dev(s0, torch.float64).requires_grad_(True)
    neg_log_posterior(s64, c64, Nd, None, m.nbar).backward()
    assert s32.grad.dtype == torch.float32
    assert rel_l2(host(s32.grad).astype(np.float64), host(s64.grad)) <= 1e-5
    # element by element: FP32 operator bar (test_gpu_operators)
    assert max_rel(host(s32.grad), host(s64.grad)) <= 2e-5
    d = np.random.default_rng(7).standard_normal(m.N.shape)
    h = 1e-5
    fp = c64.logpost_grad(dev(s0 + h * d, torch.float64), Nd, None, m.nbar, want_grad=False)[0]
    fm = c64.logpost_grad(dev(s0 - h * d, torch.float64), Nd, None, m.nbar, want_grad=False)[0]
    fd = (fp - fm) / (2 * h)
    an = float(np.sum(host(s64.grad) * d))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_map_field_backward_matches_oracle(plc):
    from paper_0911_1407_gb300.autograd import map_field
    m = mocks.make_mock(mocks.WORKLOADS["adjoint32"])
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    ref = orc.newton_krylov_map(p, tol=1e-13)
    u = np.random.default_rng(2).standard_normal(m.N.shape)
    lam_ref, lnA_ref, _ = orc.map_vjp(ref.s, u, p, rtol=1e-13)
    c = plc.Context(m.n, m.box, "fp64")
    N = dev(m.N, torch.float64).requires_grad_(True)
    ln_amp = torch.zeros((), dtype=torch.float64, device="cuda", requires_grad=True)
    s = map_field(N, ln_amp, c, m.k_tab, m.P_tab, m.mu, None, m.nbar, tol=1e-13)
    assert np.max(np.abs(host(s) - ref.s) / np.maximum(np.abs(ref.s), 1)) <= 1e-10
    (s * dev(u, torch.float64)).sum().backward()
    assert rel_l2(host(N.grad), lam_ref) <= 1e-9
    assert max_rel(host(N.grad), lam_ref) <= 1e-9
    assert abs(ln_amp.grad.item() - lnA_ref) <= 1e-9 * abs(lnA_ref)


def test_map_field_amplitude_central_difference(plc):
    """d(u . s*)/d ln A at 128^3 against a central difference with step 1e-4."""
    from paper_0911_1407_gb300.autograd import map_field
    m = mocks.make_mock(mocks.WORKLOADS["adjoint128"])
    Nd = dev(m.N, torch.float64)
    u = dev(np.random.default_rng(2).standard_normal(m.N.shape), torch.float64)
    c = plc.Context(m.n, m.box, "fp64")
    ln_amp = torch.zeros((), dtype=torch.float64, device="cuda", requires_grad=True)
    s = map_field(Nd, ln_amp, c, m.k_tab, m.P_tab, m.mu, None, m.nbar, tol=1e-11)
    (s * u).sum().backward()
    h = 1e-4
    vals = []
    for a in (h, -h):
        sa = map_field(Nd, torch.tensor(a, dtype=torch.float64, device="cuda"), c, m.k_tab,
                       m.P_tab, m.mu, None, m.nbar, tol=1e-11)
        vals.append(float((sa * u).sum()))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(ln_amp.grad.item() - fd) <= 1e-5 * abs(fd)


def test_map_field_two_amplitudes_on_one_context(plc):
    """Two MAP fields at different ln A taken on one context, then one
    backward of their sum: each gets the adjoint of its own prior (the
    second forward rescales the context's prior; the first backward must
    restore its own).  Against the oracle's VJP at each amplitude."""
    from paper_0911_1407_gb300.autograd import map_field
    m = mocks.make_mock(mocks.WORKLOADS["adjoint32"])
    rng = np.random.default_rng(11)
    u1, u2 = rng.standard_normal(m.N.shape), rng.standard_normal(m.N.shape)
    c = plc.Context(m.n, m.box, "fp64")
    outs = []
    for ln_a, u in ((0.3, u1), (-0.4, u2)):
        N = dev(m.N, torch.float64).requires_grad_(True)
        la = torch.tensor(ln_a, dtype=torch.float64, device="cuda", requires_grad=True)
        s = map_field(N, la, c, m.k_tab, m.P_tab, m.mu, None, m.nbar, tol=1e-13)
        outs.append((N, la, s, u, ln_a))
    sum((s * dev(u, torch.float64)).sum() for _, _, s, u, _ in outs).backward()
    for N, la, s, u, ln_a in outs:
        p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab * np.exp(ln_a))
        ref = orc.newton_krylov_map(p, tol=1e-13)
        assert np.max(np.abs(host(s) - ref.s) / np.maximum(np.abs(ref.s), 1)) <= 1e-10
        lam_ref, lnA_ref, _ = orc.map_vjp(ref.s, u, p, rtol=1e-13)
        assert np.max(np.abs(host(N.grad) - lam_ref)) <= 1e-9 * np.max(np.abs(lam_ref))
        assert abs(la.grad.item() - lnA_ref) <= 1e-9 * abs(lnA_ref)


def test_map_field_keeps_the_callers_dc_prior(plc):
    """inv_lambda_dc passes through the forward solve unscaled (the
    amplitude multiplies the non-DC eigenvalues only)."""
    from paper_0911_1407_gb300.autograd import map_field
    m = mocks.make_mock(mocks.WORKLOADS["adjoint32"])
    dc, ln_a = 0.05, 0.2
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab * np.exp(ln_a),
                         inv_lambda_dc=dc)
    ref = orc.newton_krylov_map(p, tol=1e-13)
    c = plc.Context(m.n, m.box, "fp64")
    la = torch.tensor(ln_a, dtype=torch.float64, device="cuda")
    s = map_field(dev(m.N, torch.float64), la, c, m.k_tab, m.P_tab, m.mu, None, m.nbar,
                  inv_lambda_dc=dc, tol=1e-13)
    assert np.max(np.abs(host(s) - ref.s) / np.maximum(np.abs(ref.s), 1)) <= 1e-10
