"""Invalid and non-finite inputs to the MAP solve (plc_newton_krylov_map).

Every case is made on the host; none can fault a GPU.

* nbar <= 0, NaN or Inf, or opts.start outside {0, 1, 2}:
  PLC_ERR_INVALID_ARG before any launch (the context's launch counters stay
  at zero).
* NaN or Inf in the selection w, or in the caller's start s0: the solve ends
  with PLC_ERR_NONFINITE, with no Newton step taken and finite statistics,
  in both drivers and both precisions.  A non-finite start reaches the
  solver through ||g0|| (the stop test's normalisation), whether the
  iteration starts there (opts.start = 0) or at the diagonal-prior start
  (opts.start = 1, where only g0 is taken at s0).
* The counts N are int32, so they hold no NaN or Inf.
"""
import math

import numpy as np
import pytest
import torch

from tests.gpu_util import dev, ensure_lib, small_mock

pytestmark = pytest.mark.gpu

NONFINITE, INVALID_ARG = 4, 1


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _ctx(plc, m, precision):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    return c


@pytest.mark.parametrize("nbar", [0.0, -1.0, float("nan"), float("inf")])
@pytest.mark.parametrize("driven", [0, 1])
def test_bad_nbar_is_refused_before_any_launch(plc, nbar, driven):
    m = small_mock(16, "uniform")
    c = _ctx(plc, m, "mixed")
    s = torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda")
    c.profile_enable(timing=False)
    r = c.newton_krylov_map(dev(m.N, torch.int32), None, nbar, s=s, device_driven=driven,
                            raise_on_fail=False)
    assert r.status == INVALID_ARG
    assert all(v[0] == 0 for v in c.profile_read().values())
    assert torch.all(s == m.mu)


@pytest.mark.parametrize("start", [-1, 3])
def test_bad_start_option_is_refused_before_any_launch(plc, start):
    m = small_mock(16, "uniform")
    c = _ctx(plc, m, "mixed")
    s = torch.full((m.n,) * 3, m.mu, dtype=torch.float64, device="cuda")
    c.profile_enable(timing=False)
    r = c.newton_krylov_map(dev(m.N, torch.int32), None, m.nbar, s=s, start=start,
                            raise_on_fail=False)
    assert r.status == INVALID_ARG
    assert all(v[0] == 0 for v in c.profile_read().values())
    assert torch.all(s == m.mu)


def _bad(where, m):
    n = m.n
    s = np.full((n,) * 3, m.mu)
    w = np.ones((n,) * 3)
    bad = {"nan": np.nan, "inf": np.inf, "-inf": -np.inf}[where.split("_")[1]]
    if where.startswith("s0"):
        s[5, 6, 7] = bad
    else:
        w[9, 2, 13] = bad
    return s, w


@pytest.mark.parametrize("where", ["s0_nan", "s0_inf", "s0_-inf", "w_nan", "w_inf", "w_-inf"])
@pytest.mark.parametrize("start", [0, 1])
@pytest.mark.parametrize("driven", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_finite_input_ends_the_solve(plc, where, start, driven, precision):
    m = small_mock(16, "uniform")
    c = _ctx(plc, m, precision)
    s0, w = _bad(where, m)
    r = c.newton_krylov_map(dev(m.N, torch.int32), dev(w, torch.float64), m.nbar,
                            s=dev(s0, torch.float64), start=start, device_driven=driven,
                            tol=1e-6, raise_on_fail=False)
    assert r.status == NONFINITE
    st = r.stats
    assert st["newton_iters"] == 0 and st["cg_iters"] == 0
    assert math.isfinite(st["grad_rel"])
    # the context stays usable: a clean solve on it converges
    ok = c.newton_krylov_map(dev(m.N, torch.int32), None, m.nbar, tol=1e-6, device_driven=driven)
    assert ok.status == 0 and ok.stats["grad_rel"] < 1e-6
