"""Edge and degenerate cases of the MAP solve on the GPU.

* No counts at all (N = 0): the MAP balances the prior against the expected
  counts alone; parity with the oracle.
* Nothing observed (w = 0, N = 0): g(mu) = 0, so the solve stops at s = mu
  with no Newton step, in both drivers.
* One cell with a very large count next to empty cells: parity with the
  oracle (a sharp, high peak of s).
* The largest grid the library takes, 512^3 (Stockham FP32 passes): no
  oracle at that size, so properties that hold at any size -- the FP64 GPU
  gradient norm at the returned MAP, and the DC balance of the flat prior on
  the mean, |sum nbar w e^s - sum N| <= sqrt(n^3) ||g|| (Cauchy-Schwarz on
  the DC component of g).
"""
import math

import numpy as np
import pytest
import torch

from oracle import plc as orc
from paper_0911_1407_gb300 import mocks
from tests.gpu_util import dev, ensure_lib, host, small_mock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plc():
    return ensure_lib()


def _ctx(plc, m, precision):
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu)
    return c


def _problem(m, N=None, w=None):
    return orc.make_problem(m.N if N is None else N, m.w if w is None else w, m.nbar, m.mu, m.n,
                            m.box, m.k_tab, m.P_tab)


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_no_counts(plc, precision, bar):
    """With a proper prior on the mean (inv_lambda_dc > 0) the posterior of
    empty data has a mode, with its mean below the prior mean."""
    m = small_mock(16, "radial_masked", sigma=1.0, nbar=1.5)
    N = np.zeros_like(m.N)
    p = orc.make_problem(N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab, inv_lambda_dc=1.0)
    ref = orc.newton_krylov_map(p, tol=1e-12)
    assert ref.converged
    c = plc.Context(m.n, m.box, precision)
    c.set_prior(m.k_tab, m.P_tab, m.mu, 1.0)
    r = c.newton_krylov_map(dev(N, torch.int32), dev(m.w, torch.float64), m.nbar,
                            tol=1e-12 if precision == "fp64" else 1e-6)
    s = host(r.s)
    assert np.max(np.abs(s - ref.s) / np.maximum(np.abs(ref.s), 1.0)) <= bar
    # the DC component of g = 0: inv_lambda_dc mean(s - mu) = -mean(nbar w e^s) < 0
    assert s.mean() < m.mu


@pytest.mark.parametrize("driven", [0, 1])
def test_no_counts_with_a_flat_mean_prior_has_no_mode(plc, driven):
    """With the flat prior on the mean (c4) and no counts there is no mode:
    the mean of s runs off to -inf while ||g|| = ||nbar w e^s|| shrinks, so
    the relative stop test ends the solve far below mu (the oracle does the
    same); the solve must end, with finite values."""
    m = small_mock(16, "radial_masked", sigma=1.0, nbar=1.5)
    c = _ctx(plc, m, "mixed")
    r = c.newton_krylov_map(torch.zeros((m.n,) * 3, dtype=torch.int32, device="cuda"),
                            dev(m.w, torch.float64), m.nbar, tol=1e-6, device_driven=driven,
                            raise_on_fail=False)
    assert r.status in (0, 3)
    assert torch.isfinite(r.s).all() and float(r.s.mean()) < m.mu - 10.0


@pytest.mark.parametrize("driven", [0, 1])
def test_nothing_observed_stops_at_the_prior_mean(plc, driven):
    m = small_mock(16, "uniform", sigma=1.0, nbar=1.5)
    c = _ctx(plc, m, "mixed")
    N = torch.zeros((m.n,) * 3, dtype=torch.int32, device="cuda")
    w = torch.zeros((m.n,) * 3, dtype=torch.float64, device="cuda")
    r = c.newton_krylov_map(N, w, m.nbar, tol=1e-6, device_driven=driven)
    assert r.status == 0 and r.stats["newton_iters"] == 0 and r.stats["cg_iters"] == 0
    assert r.stats["grad_rel"] == 0.0
    assert torch.all(r.s == m.mu)


@pytest.mark.parametrize("precision,bar", [("fp64", 2e-7), ("mixed", 1e-4)])
def test_one_very_large_count(plc, precision, bar):
    """One cell dominates ||g0|| (~2e4), so the relative stop test 1e-12
    leaves an absolute gradient of ~2e-8 and the MAP is fixed only to about
    that over the smallest Hessian eigenvalue (the oracle's own MAPs at 1e-12
    and 1e-14 differ by 4.5e-8): the FP64 bar is set from that bound."""
    m = small_mock(16, "uniform", sigma=1.0, nbar=0.2)
    N = np.zeros_like(m.N)
    N[3, 7, 11] = 20000
    N[3, 7, 12] = 1
    ref = orc.newton_krylov_map(_problem(m, N=N), tol=1e-12)
    assert ref.converged
    c = _ctx(plc, m, precision)
    # the mixed form is driven to 1e-10 (its FP64 phase): at 1e-6 the same
    # bound leaves ~2e-2 in the background cells
    r = c.newton_krylov_map(dev(N, torch.int32), None, m.nbar,
                            tol=1e-12 if precision == "fp64" else 1e-10)
    s = host(r.s)
    assert np.max(np.abs(s - ref.s) / np.maximum(np.abs(ref.s), 1.0)) <= bar
    assert s[3, 7, 11] == s.max()


def _large_counts(n, box, nbar, sigma, seed):
    """Seeded counts at a size the host mock generator would take minutes
    for: a Gaussian-smoothed white-noise log-density of standard deviation
    about sigma on the device, Poisson counts from torch (test input only;
    nothing here is compared with the oracle)."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((n, n, n), generator=g, device="cuda", dtype=torch.float32)
    f = torch.fft.fftfreq(n, d=box / n, device="cuda") * 2 * math.pi
    k2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, : n // 2 + 1] ** 2
    G = torch.fft.irfftn(torch.fft.rfftn(x) * torch.exp(-0.5 * k2 * 8.0 ** 2), s=(n, n, n))
    G = G * (sigma / G.std())
    N = torch.poisson(nbar * torch.exp(G - 0.5 * sigma ** 2), generator=g).to(torch.int32)
    return N


def test_largest_grid_512(plc):
    n, box, nbar, sigma = 512, 1000.0, 1.0, 1.8
    A = mocks.amplitude_for_sigma(n, box, sigma)
    k, P = mocks.pk_table(n, box, A)
    mu = -0.5 * sigma ** 2
    Nd = _large_counts(n, box, nbar, sigma, seed=5)
    c = plc.Context(n, box, "mixed")
    c.set_prior(k, P, mu)
    r = c.newton_krylov_map(Nd, None, nbar, tol=1e-6)
    assert r.status == 0 and r.stats["grad_rel"] < 1e-6
    # the FP64 gradient at the returned MAP, by the FP64 operators
    c64 = plc.Context(n, box, "fp64")
    c64.set_prior(k, P, mu)
    _, g = c64.logpost_grad(r.s, Nd, None, nbar)
    _, g0 = c64.logpost_grad(torch.full_like(r.s, mu), Nd, None, nbar)
    gn, g0n = float(g.norm()), float(g0.norm())
    assert gn / g0n < 1e-6
    assert abs(gn / g0n - r.stats["grad_rel"]) <= 1e-3 * r.stats["grad_rel"]
    mass = float((nbar * torch.exp(r.s)).sum())
    assert abs(mass - float(Nd.double().sum())) <= math.sqrt(n ** 3) * gn * (1 + 1e-9)
