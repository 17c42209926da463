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
    L.md_host_two_sum.argtypes = [C.c_int, C.c_long, dp, dp, dp, dp]

    def run(p, op, a, b, c=None):
        a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
        c = np.zeros_like(a) if c is None else np.ascontiguousarray(c).copy()
        L.md_host_op(p, OPS[op], a.shape[1], a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                     c.ctypes.data_as(dp))
        return c
    run.lib, run.dp = L, dp
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


def _two_sum_inputs(rng, n):
    """Pairs that exercise every path of the error-free sum: mixed
    magnitudes, near and exact cancellation, gaps beyond 53 bits and beyond
    64, halfway cases (b = +-ulp(a)/2, 3 ulp(a)/2), subnormals, signed zeros
    and magnitudes near overflow."""
    def rnd(k, lo, hi):
        m = 1.0 + rng.integers(0, 2 ** 52, k) * 2.0 ** -52
        v = np.ldexp(m, rng.integers(lo, hi + 1, k))
        return np.where(rng.integers(0, 2, k) == 1, -v, v)
    k = n // 8
    parts = []
    parts.append((rnd(k, -30, 30), rnd(k, -30, 30)))
    a = rnd(k, -5, 5)
    parts.append((a, -a * (1 + rnd(k, -60, -40))))
    parts.append((rnd(k, -1074, -1000), rnd(k, -1074, -1000)))
    parts.append((rnd(k, -100, 100), rnd(k, -300, 300)))
    a = rnd(k, -10, 10)
    h = np.ldexp(1.0, np.frexp(a)[1] - 54)
    parts.append((np.concatenate([a, a, a]), np.concatenate([h, -h, 3 * h])))
    parts.append((rnd(k, 1000, 1022), rnd(k, 900, 1022)))
    z = rnd(k, -20, 20)
    zeros = np.array([0.0, -0.0])[rng.integers(0, 2, k)]
    parts.append((np.concatenate([z, zeros, zeros]), np.concatenate([zeros, z, zeros[::-1]])))
    bits = rng.integers(0, 2 ** 63, (2, k), dtype=np.int64).view(np.float64)
    ok = np.isfinite(bits[0]) & np.isfinite(bits[1])
    parts.append((bits[0][ok], bits[1][ok]))
    a = np.concatenate([p[0] for p in parts] + [p[1] for p in parts])
    b = np.concatenate([p[1] for p in parts] + [p[0] for p in parts])
    return a, b


def test_two_sum_forms_are_exact_and_agree(harness):
    """Both two_sum forms give s = fl(a + b) and the exact error (Knuth's
    TwoSum evaluated in numpy is the reference value), bit for bit the same
    in either form, signed zeros included, for finite sums."""
    rng = np.random.default_rng(7)
    a, b = _two_sum_inputs(rng, 400000)
    L, dp = harness.lib, harness.dp
    out = {}
    for form in (0, 1):
        s = np.zeros_like(a)
        e = np.zeros_like(a)
        L.md_host_two_sum(form, a.size, a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                          s.ctypes.data_as(dp), e.ctypes.data_as(dp))
        out[form] = (s, e)
    with np.errstate(over="ignore", invalid="ignore"):
        s_ref = a + b
        bb = s_ref - a
        e_ref = (a - (s_ref - bb)) + (b - bb)
    fin = np.isfinite(s_ref)
    assert fin.sum() > 0.95 * a.size
    for form in (0, 1):
        s, e = out[form]
        assert np.array_equal(s[fin].view(np.int64), s_ref[fin].view(np.int64))
        assert np.array_equal(e[fin], e_ref[fin])
    assert np.array_equal(out[0][1][fin].view(np.int64), out[1][1][fin].view(np.int64))
    # an overflowing sum gives a non-finite error in both forms
    assert not np.isfinite(out[0][1][~fin]).any() and not np.isfinite(out[1][1][~fin]).any()
