"""The warp-parallel digit scalars of csrc/fxw.cuh (the panel's Householder
scalars and per-reflector products spread over one warp, digit k in lane k)
against their one-thread namesakes of csrc/fx.cuh, digit for digit, on random
sign-consistent inputs in every precision: products, sums with cancellation
and disjoint windows, Newton reciprocals and inverse square roots, the three
kinds of Householder scalars, conversions from doubles and to and from the
fixed-point column format, bit shifts and wide dot-product accumulators,
multiple doubles to digits, and the panels' two-step Householder scalars
(lanes sharing the double double conversions) against the one-thread forms.  The
scalar routines are pinned to exact rational arithmetic by test_fx_host.py."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OPS = ["mul", "add", "sub", "recip", "rsqrt", "house", "from_double", "fixed", "shift_bits", "from_acc",
       "from_md", "panel_house"]


@pytest.fixture(scope="module")
def fxw():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = os.path.join(tempfile.mkdtemp(), "fxw_check.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-o", out,
                    os.path.join(ROOT, "tests", "harness", "fxw_check.cu")], check=True)
    L = C.CDLL(out)
    L.fxw_check.argtypes = [C.c_int, C.c_int, C.c_ulonglong, C.POINTER(C.c_int)]
    L.fxw_check.restype = C.c_int
    return L


@pytest.mark.parametrize("p", [2, 4, 8])
def test_warp_digits_match_scalar(fxw, p):
    bad = (C.c_int * len(OPS))()
    rc = fxw.fxw_check(p, 6000, 1000 + p, bad)
    assert rc == 0
    assert list(bad) == [0] * len(OPS), dict(zip(OPS, list(bad)))
