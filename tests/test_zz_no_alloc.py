"""The allocation-free Hessian-vector product against the context-based one.

plc_hessvec_noalloc serves callers that cannot call cudaMalloc (device
memory reserved up front by an allocator they do not own, code that forbids
allocation after start-up, plug-ins without allocations of their own).  It
must give what plc_hessvec gives on an FP64 context, within the FP64 bar of
the operator tests (1e-12 relative), on consecutive calls that reuse its
static scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from tests.gpu_util import ensure_lib, pk_table_for

pytestmark = pytest.mark.gpu


def _call(lib, n, box, k, P, dc, s, w, nbar, v, out):
    DP = ctypes.POINTER(ctypes.c_double)
    k = np.ascontiguousarray(k, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return lib.plc_hessvec_noalloc(n, box, k.ctypes.data_as(DP), P.ctypes.data_as(DP), k.size, dc,
                                   ptr(s), ptr(w), nbar, ptr(v), ptr(out),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_hessvec_matches_context_hessvec_twice():
    plc = ensure_lib()
    lib = plc.load()
    rng = np.random.default_rng(11)
    # two calls in a row: different sizes, tables, fields; the second call
    # runs on scratch that still holds the first call's contents
    for n, box, dc, with_w in ((48, 300.0, 0.0, True), (64, 420.0, 0.21, False)):
        k, P = pk_table_for(n, box, seed=n)
        s = torch.from_numpy(-0.5 + 0.6 * rng.standard_normal((n,) * 3)).cuda()
        w = torch.from_numpy(rng.uniform(0.1, 1.0, (n,) * 3)).cuda() if with_w else None
        v = torch.from_numpy(rng.standard_normal((n,) * 3)).cuda()
        out = torch.full((n,) * 3, float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, n, box, k, P, dc, s, w, 1.3, v, out) == 0
        with plc.Context(n, box, "fp64") as c:
            c.set_prior(k, P, -0.5, dc)
            ref = c.hessvec(s, w, 1.3, v)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= 1e-12, (n, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    plc = ensure_lib()
    lib = plc.load()
    n, box = 96, 500.0
    k, P = pk_table_for(n, box)
    f = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
    assert _call(lib, n, box, k, P, 0.0, f, None, 1.0, f, f) == 1
    assert b"64" in lib.plc_last_error(None)
