"""The allocation-free Hessian-vector product.

plc_hessvec_noalloc serves callers that cannot call cudaMalloc (device
memory reserved up front by an allocator they do not own, code that forbids
allocation after start-up, plug-ins without allocations of their own).  It
must give what the FP64 oracle's H v gives and what plc_hessvec gives on an
FP64 context, within the FP64 bar of the operator tests (1e-12 of the
peak element), on consecutive calls that reuse its static scratch.

The file's name makes pytest collect it last, so that a run stopping at the
first failure has run every other test before this one.  The first call on
a device (the scratch address lookup) is also exercised in a fresh process.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import plc as orc
from tests.gpu_util import ensure_lib, pk_table_for

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _call(lib, n, box, k, P, dc, s, w, nbar, v, out):
    DP = ctypes.POINTER(ctypes.c_double)
    k = np.ascontiguousarray(k, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return lib.plc_hessvec_noalloc(n, box, k.ctypes.data_as(DP), P.ctypes.data_as(DP), k.size, dc,
                                   ptr(s), ptr(w), nbar, ptr(v), ptr(out),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _oracle_hv(n, box, k, P, dc, s, w, nbar, v):
    p = orc.make_problem(np.zeros((n,) * 3, np.int32), w, nbar, 0.0, n, box, k, P, dc)
    return orc.hessvec(s, v, p)


def test_noalloc_hessvec_matches_oracle_and_context_hessvec_twice():
    plc = ensure_lib()
    lib = plc.load()
    rng = np.random.default_rng(11)
    # two calls in a row: different sizes, tables, fields; the second call
    # runs on scratch that still holds the first call's contents
    for n, box, dc, with_w in ((48, 300.0, 0.0, True), (64, 420.0, 0.21, False)):
        k, P = pk_table_for(n, box, seed=n)
        s_h = -0.5 + 0.6 * rng.standard_normal((n,) * 3)
        w_h = rng.uniform(0.1, 1.0, (n,) * 3) if with_w else None
        v_h = rng.standard_normal((n,) * 3)
        s = torch.from_numpy(s_h).cuda()
        w = torch.from_numpy(w_h).cuda() if with_w else None
        v = torch.from_numpy(v_h).cuda()
        out = torch.full((n,) * 3, float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, n, box, k, P, dc, s, w, 1.3, v, out) == 0
        with plc.Context(n, box, "fp64") as c:
            c.set_prior(k, P, -0.5, dc)
            ref = c.hessvec(s, w, 1.3, v)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= 1e-12, (n, err)
        hv = _oracle_hv(n, box, k, P, dc, s_h, w_h, 1.3, v_h)
        err_o = float(np.max(np.abs(out.cpu().numpy() - hv)) / np.max(np.abs(hv)))
        assert err_o <= 1e-12, (n, err_o)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    plc = ensure_lib()
    lib = plc.load()
    n, box = 96, 500.0
    k, P = pk_table_for(n, box)
    f = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
    assert _call(lib, n, box, k, P, 0.0, f, None, 1.0, f, f) == 1
    assert b"64" in lib.plc_last_error(None)


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from tests.test_zz_no_alloc import _call, _oracle_hv
from tests.gpu_util import pk_table_for
import paper_0911_1407_gb300 as plc
lib = plc.load()
n, box, dc = 32, 200.0, 0.05
k, P = pk_table_for(n, box, seed=3)
rng = np.random.default_rng(4)
s_h, v_h = -0.3 + 0.5 * rng.standard_normal((n,) * 3), rng.standard_normal((n,) * 3)
out = torch.full((n,) * 3, float("nan"), dtype=torch.float64, device="cuda")
st = _call(lib, n, box, k, P, dc, torch.from_numpy(s_h).cuda(), None, 0.8,
           torch.from_numpy(v_h).cuda(), out)
assert st == 0, lib.plc_last_error(None)
torch.cuda.synchronize()
hv = _oracle_hv(n, box, k, P, dc, s_h, None, 0.8, v_h)
err = float(np.max(np.abs(out.cpu().numpy() - hv)) / np.max(np.abs(hv)))
assert err <= 1e-12, err
print("fresh-process noalloc ok", err)
"""


def test_noalloc_first_call_in_a_fresh_process():
    """The first call on a device (scratch address lookup, then the passes)
    in a process that has run nothing else of the library."""
    ensure_lib()
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "fresh-process noalloc ok" in r.stdout
