"""The device multiple-double arithmetic (csrc/md.cuh) compiled for the host
and checked against the oracle's exact-then-rounded operations on the CPU.

md.cuh is host/device code; on the host the intrinsics become plain IEEE
operations and the harness is built with -ffp-contract=off, so the same
sequence of roundings runs as on the GPU.  Covers random operands, exact and
near-exact cancellation (which once left a zero leading limb in front of the
value and stalled the square root), very different magnitudes, and the limb
normalisation of every result."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "fma": 4, "sqrt": 5}
BOUND = {2: 2.0 ** -100, 4: 2.0 ** -204, 8: 2.0 ** -410}


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = os.path.join(tempfile.mkdtemp(), "md_host.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
                    "-o", out, os.path.join(ROOT, "tests", "harness", "md_host.cu")], check=True)
    L = C.CDLL(out)
    dp = C.POINTER(C.c_double)
    L.md_host_op.argtypes = [C.c_int, C.c_int, C.c_long, dp, dp, dp]

    def run(p, op, a, b, c=None):
        a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
        c = np.zeros_like(a) if c is None else np.ascontiguousarray(c).copy()
        L.md_host_op(p, OPS[op], a.shape[1], a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                     c.ctypes.data_as(dp))
        return c
    return run


def draw(rng, p, n, lo=-20, hi=20):
    x = np.zeros((p, n))
    x[0] = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(lo, hi, n)
    for i in range(1, p):
        x[i] = x[i - 1] * 2.0 ** -54 * rng.uniform(-1, 1, n)
    return x


def reference(op, a, b, c):
    n = a.shape[1]
    out = np.zeros_like(a)
    for i in range(n):
        if op == "fma":
            out[:, i] = oracle.add(c[:, i], oracle.mul(a[:, i], b[:, i]))
        elif op == "sqrt":
            out[:, i] = oracle.sqrt(a[:, i])
        else:
            out[:, i] = getattr(oracle, op)(a[:, i], b[:, i])
    return out


def check(p, op, a, b, c, got):
    ref = reference(op, a, b, c)
    d = np.abs(oracle.diff(got, ref))
    scale = {"add": np.abs(a[0]) + np.abs(b[0]), "sub": np.abs(a[0]) + np.abs(b[0]),
             "mul": np.abs(a[0] * b[0]), "div": np.abs(a[0] / np.where(b[0] == 0, 1, b[0])),
             "fma": (np.abs(c[0]) if c is not None else 0) + np.abs(a[0] * b[0]),
             "sqrt": np.sqrt(np.abs(a[0]))}[op]
    worst = float(np.max(d / np.where(scale > 0, scale, 1.0)))
    assert worst <= BOUND[p], (op, p, worst)
    # leading limb nonzero whenever the value is, no zero limb before a nonzero one
    nz = got != 0
    for i in range(p - 1):
        assert not np.any(~nz[i] & nz[i + 1]), (op, p, "zero limb in front of a nonzero one")


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "fma", "sqrt"])
def test_random_operands(harness, p, op):
    rng = np.random.default_rng(hash((p, op)) % 2 ** 32)
    n = 400
    a, b, c = draw(rng, p, n), draw(rng, p, n), draw(rng, p, n)
    if op == "sqrt":
        a = a * np.sign(a[0])
    got = harness(p, op, a, b, c if op == "fma" else None)
    check(p, op, a, b, c if op == "fma" else None, got)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_cancellation(harness, p):
    rng = np.random.default_rng(p)
    n = 400
    a = draw(rng, p, n)
    b = -a.copy()
    b[p - 1] += a[p - 1] * 2.0 ** -20 * rng.uniform(-1, 1, n)       # near-exact cancellation
    b[:, : n // 4] = -a[:, : n // 4]                                  # exact cancellation
    check(p, "add", a, b, None, harness(p, "add", a, b))
    # c - x*x with x the md square root of c: the residual of a Newton step
    c = np.abs(draw(rng, p, n)) * 0 + draw(rng, p, n)
    c = c * np.sign(c[0])
    x = np.stack([oracle.sqrt(c[:, i]) for i in range(n)], axis=1)
    x[p // 2:] = 0.0
    check(p, "fma", -x, x, c, harness(p, "fma", -x, x, c))


@pytest.mark.parametrize("p", [2, 4, 8])
def test_far_apart_magnitudes(harness, p):
    rng = np.random.default_rng(10 + p)
    n = 300
    a = draw(rng, p, n, 0, 1)
    b = draw(rng, p, n, -300, -150)
    for op in ("add", "sub", "mul", "div"):
        check(p, op, a, b, None, harness(p, op, a, b))
