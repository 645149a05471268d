"""The C-ABI library builds, loads and exports every function plc.h declares.

Runs without a GPU: only calls that validate arguments before touching CUDA
(plc_create with an invalid size, plc_default_opts, plc_status_string) are
made.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_0911_1407_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("plc_logpost_grad", "plc_hessvec", "plc_newton_krylov_map", "plc_map_vjp",
                 "plc_prior_apply", "plc_create", "plc_set_prior"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in plc.h but not exported"


def test_binding_covers_every_symbol():
    from paper_0911_1407_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    lib.plc_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.c_void_p]
    for bad_n in (0, 7, 10, 14, 1024):
        assert lib.plc_create(ctypes.byref(h), bad_n, 100.0, 0, None) == 1
    assert lib.plc_create(ctypes.byref(h), 16, -1.0, 0, None) == 1
    assert lib.plc_create(ctypes.byref(h), 16, 100.0, 5, None) == 1
    lib.plc_status_string.restype = ctypes.c_char_p
    assert lib.plc_status_string(3) == b"PLC_ERR_NOT_CONVERGED"
    from paper_0911_1407_gb300._lib import Opts
    o = Opts()
    assert lib.plc_default_opts(ctypes.byref(o)) == 0
    assert o.tol == 1e-6 and o.precond == 1 and o.max_cg == 1000
    assert o.device_driven == 1 and o.mixed_switch == 1e-6


def test_batch_validation_without_gpu(lib):
    b = ctypes.c_void_p()
    P = ctypes.c_void_p
    lib.plc_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int]
    assert lib.plc_batch_create(None, None, 1) == 1
    assert lib.plc_batch_create(ctypes.byref(b), None, 1) == 1
    arr = (P * 2)(None, None)
    assert lib.plc_batch_create(ctypes.byref(b), arr, 2) == 1     # NULL context
    assert lib.plc_batch_create(ctypes.byref(b), arr, 0) == 1     # empty batch
    lib.plc_batch_map.argtypes = [P] * 8
    assert lib.plc_batch_map(None, None, None, None, None, None, None, None) == 1
    lib.plc_batch_destroy.argtypes = [P]
    assert lib.plc_batch_destroy(None) == 0


def test_bias_validation_without_gpu(lib):
    P = ctypes.c_void_p
    D = ctypes.c_double
    DP = ctypes.POINTER(D)
    lib.plc_set_bias.argtypes = [P, DP, DP, ctypes.c_int, D]
    k = (D * 2)(0.1, 1.0)
    b = (D * 2)(1.2, 1.5)
    assert lib.plc_set_bias(None, k, b, 2, 1.0) == 1
    lib.plc_bias_map.argtypes = [P] * 3 + [D] + [P] * 3
    assert lib.plc_bias_map(None, None, None, 1.0, None, None, None) == 1
    lib.plc_bias_logpost_grad.argtypes = [P] * 4 + [D, P, P]
    assert lib.plc_bias_logpost_grad(None, None, None, None, 1.0, None, None) == 1
    lib.plc_bias_hessvec.argtypes = [P] * 4 + [D, P, P]
    assert lib.plc_bias_hessvec(None, None, None, None, 1.0, None, None) == 1


def test_header_is_plain_c_and_links(lib):
    """include/plc.h compiles as C99 with -pedantic, and a C program links
    against libplc.so and calls a host-only entry point.  Built in the
    package's (ignored) build directory."""
    import pathlib
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    work = pathlib.Path(ROOT) / "paper_0911_1407_gb300" / "_build" / "ctest"
    work.mkdir(parents=True, exist_ok=True)
    src = work / "t.c"
    src.write_text('#include "plc.h"\n'
                   'int main(void) { plc_opts o; if (plc_default_opts(&o) != PLC_OK) return 2;\n'
                   '  return (o.max_newton > 0 && o.tol > 0.0 && o.device_driven == 1) ? 0 : 1; }\n')
    libdir = os.path.join(ROOT, "paper_0911_1407_gb300")
    exe = work / "t"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lplc",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    assert subprocess.run([str(exe)]).returncode == 0
