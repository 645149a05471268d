"""The device-driven solve (one CUDA graph launch per solve, decisions in
control kernels) against the host-driven one, and batches of independent
solves in one graph launch.

Both drivers launch the same kernels with the same arguments in the same
order on the same data (the host driver only adds CG launches that exit at
once on the done flag), so their results must agree bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import plc as orc
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host, small_mock

pytestmark = pytest.mark.gpu

ITER_KEYS = ("newton_iters", "cg_iters", "hv_count", "grad_evals", "grad_ffts", "grad_ffts_fp64")


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _ctx(plc, m, precision):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    return c


def _solve(c, m, driven, **kw):
    s = torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda")
    r = c.newton_krylov_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, s=s,
                            device_driven=driven, raise_on_fail=False, **kw)
    return r


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_start_off_the_prior_mean(plc, precision):
    """A start point off mu takes the FFT gradient there for ||g0|| (the IF
    node of the device-driven graph); both drivers agree bit for bit, and
    a start at mu needs no transform for ||g0||."""
    m = small_mock(32, "radial_masked", sigma=1.2, nbar=1.0)
    c = _ctx(plc, m, precision)
    s0 = torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda")
    s0[5, 6, 7] += 0.25
    out = []
    for driven in (0, 1):
        s = s0.clone()
        r = c.newton_krylov_map(dev(m.N, torch.int32), dev(m.w, torch.float64), m.nbar, s=s,
                                tol=1e-6, device_driven=driven)
        out.append(r)
    for k in ITER_KEYS:
        assert out[0].stats[k] == out[1].stats[k], k
    assert torch.equal(out[0].s, out[1].s)
    at_mean = _solve(c, m, 1, tol=1e-6)
    assert out[1].stats["grad_ffts"] == at_mean.stats["grad_ffts"] + 1
    assert out[1].stats["g0_norm"] != at_mean.stats["g0_norm"]


def test_cached_graphs_for_alternating_buffers(plc):
    """Solves that alternate between buffer sets (and more sets than the
    cache holds) relaunch or recapture the right graph: every result equals
    the host-driven one bit for bit."""
    m = small_mock(32, "radial_masked", sigma=1.2, nbar=1.0)
    c = _ctx(plc, m, "mixed")
    ref = _solve(c, m, 0, tol=1e-6)
    sets = [(dev(m.N, torch.int32), dev(m.w, torch.float64),
             torch.empty((m.n,) * 3, dtype=torch.float64, device="cuda")) for _ in range(6)]
    for k in [0, 1, 0, 1, 2, 3, 4, 5, 0, 1, 5]:
        N, w, s = sets[k]
        s.fill_(m.mu)
        r = c.newton_krylov_map(N, w, m.nbar, s=s, tol=1e-6, device_driven=1)
        assert torch.equal(s, ref.s), k
        assert r.stats["cg_iters"] == ref.stats["cg_iters"]


@pytest.mark.parametrize("key,precision,tol", [("plain32", "fp64", 1e-12), ("plain32", "mixed", 1e-6),
                                               ("sel48", "mixed", 1e-6), ("sel48", "fp64", 1e-10),
                                               ("production256", "mixed", 1e-6)])
def test_device_driven_equals_host_driven(plc, key, precision, tol):
    if key == "sel48":
        m = small_mock(48, "radial_masked", sigma=1.5, nbar=0.5)
    else:
        m = mocks.make_mock(mocks.WORKLOADS[key])
    c = _ctx(plc, m, precision)
    rh = _solve(c, m, 0, tol=tol)
    rd = _solve(c, m, 1, tol=tol)
    assert rh.status == 0 and rd.status == 0
    for k in ITER_KEYS:
        assert rh.stats[k] == rd.stats[k], k
    assert rh.stats["grad_rel"] == rd.stats["grad_rel"]
    assert torch.equal(rh.s, rd.s)
    assert rd.stats["kernels"] > 5 * rd.stats["cg_iters"]
    # relaunching the cached graph gives the same again
    rd2 = _solve(c, m, 1, tol=tol)
    assert torch.equal(rd.s, rd2.s) and rd2.stats["cg_iters"] == rd.stats["cg_iters"]


def test_device_driven_iteration_cap_and_resume(plc):
    m = mocks.make_mock(mocks.WORKLOADS["plain32"])
    c = _ctx(plc, m, "fp64")
    Nd = dev(m.N, torch.int32)
    s = torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda")
    r1 = c.newton_krylov_map(Nd, None, m.nbar, s=s, tol=1e-12, max_newton=2, raise_on_fail=False)
    assert r1.status == 3 and r1.stats["newton_iters"] == 2
    r2 = c.newton_krylov_map(Nd, None, m.nbar, s=r1.s, tol=1e-12, g0_norm=r1.stats["g0_norm"])
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    ref = orc.newton_krylov_map(p, tol=1e-12)
    assert np.max(np.abs(host(r2.s) - ref.s) / np.maximum(np.abs(ref.s), 1)) <= 1e-10


def test_batch_equals_one_by_one(plc):
    """Mocks of uneven sizes (four-step and Stockham lengths, both precisions,
    with and without selection) in one graph launch."""
    ms = [small_mock(32, "uniform", sigma=1.0, nbar=2.0, seed=3),
          small_mock(48, "radial_masked", sigma=1.3, nbar=0.7, seed=4),
          small_mock(64, "uniform", sigma=1.6, nbar=0.3, seed=5),
          small_mock(24, "radial_masked", sigma=0.9, nbar=1.5, seed=6)]
    precs = ["mixed", "fp64", "mixed", "fp64"]
    cs = [_ctx(plc, m, p) for m, p in zip(ms, precs)]
    singles = [_solve(c, m, 1, tol=1e-8) for c, m in zip(cs, ms)]
    Ns = [dev(m.N, torch.int32) for m in ms]
    ws = [dev(m.w, torch.float64) for m in ms]
    ss = [torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda") for m in ms]
    b = plc.Batch(cs)
    st, stats = b.map(Ns, ws, [m.nbar for m in ms], ss, tol=1e-8)
    assert st == 0
    for r, s, bst in zip(singles, ss, stats):
        assert torch.equal(r.s, s)
        for k in ITER_KEYS:
            assert r.stats[k] == bst[k], k
    # a second launch of the cached batch graph from the same start
    for s, m in zip(ss, ms):
        s.fill_(m.mu)
    st2, stats2 = b.map(Ns, ws, [m.nbar for m in ms], ss, tol=1e-8)
    assert st2 == 0
    for r, s in zip(singles, ss):
        assert torch.equal(r.s, s)


def test_batch_start_at_mean_reads_no_start_arrays(plc):
    """opts.start = 2 in a batch: start arrays full of NaN give the same MAPs,
    bit for bit, and the same iterations as start = 1 from arrays filled
    with mu."""
    ms = [small_mock(32, "uniform", sigma=1.0, nbar=2.0, seed=3),
          small_mock(48, "radial_masked", sigma=1.3, nbar=0.7, seed=4),
          small_mock(24, "radial_masked", sigma=0.9, nbar=1.5, seed=6)]
    cs = [_ctx(plc, m, p) for m, p in zip(ms, ["mixed", "fp64", "mixed"])]
    Ns = [dev(m.N, torch.int32) for m in ms]
    ws = [dev(m.w, torch.float64) for m in ms]
    nb = [m.nbar for m in ms]
    s1 = [torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda") for m in ms]
    s2 = [torch.full((m.n,) * 3, float("nan"), dtype=torch.float64, device="cuda") for m in ms]
    b = plc.Batch(cs)
    st1, stats1 = b.map(Ns, ws, nb, s1, tol=1e-8, start=1)
    st2, stats2 = b.map(Ns, ws, nb, s2, tol=1e-8, start=2)   # captured again: new key
    assert st1 == 0 and st2 == 0
    for a, c, x, y in zip(s1, s2, stats1, stats2):
        assert torch.equal(a, c)
        for k in ITER_KEYS:
            assert x[k] == y[k], k


@pytest.mark.parametrize("tol", [4e-7, 3e-7, 2e-7, 1.5e-7, 1e-7])
def test_drivers_agree_near_the_fp32_floor(plc, tol):
    """Mixed solves whose tolerance sits near the FP32 gradient's rounding
    floor: at the switch the FP64 gradient's sums are taken first when the
    FP32 gradient passes the test, and the full FP64 gradient (and more
    Newton steps) follows when the FP64 sums fail it.  Whichever branch a
    tolerance takes, both drivers take it identically and the solve meets
    its tolerance on the FP64 gradient."""
    m = mocks.make_mock(mocks.WORKLOADS["plain32"])
    c = _ctx(plc, m, "mixed")
    rh = _solve(c, m, 0, tol=tol)
    rd = _solve(c, m, 1, tol=tol)
    assert rh.status == 0 and rd.status == 0
    for k in ITER_KEYS:
        assert rh.stats[k] == rd.stats[k], k
    assert torch.equal(rh.s, rd.s)
    assert rd.stats["grad_rel"] < tol and rd.stats["grad_ffts_fp64"] >= 1
