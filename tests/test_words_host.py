"""The split products' exact epilogue (csrc/words.cuh) compiled for the host:
a multiword integer sum_g W_g 2^(32 g + e0), plus an md value added exactly
on the 2^e0 grid, rounded toward zero to P limbs greedily (limb 0 the leading
53 bits of the magnitude, each next limb the leading 53 bits of what is
left).  Checked bit for bit against the same definition in Python integers,
on random words of both signs near their 2^56 bound, carries across every
word boundary, exact cancellation, values with long zero runs between limbs,
and md addends below, inside and above the words' own range."""
import ctypes as C
import os
import random
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GW = {2: 7, 4: 10, 8: 17}


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = os.path.join(tempfile.mkdtemp(), "words_host.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", "-o", out,
                    os.path.join(ROOT, "tests", "harness", "words_host.cu")], check=True)
    L = C.CDLL(out)
    L.words_host_to_md.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_int,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
    return L


def grid(x, e0):
    """The double x truncated toward zero onto the grid 2^e0, in units 2^e0."""
    f = Fraction(x) / Fraction(2) ** e0
    return int(f) if f >= 0 else -int(-f)


def expected(p, words, e0, negate, c):
    total = sum(w << (32 * g) for g, w in enumerate(words))
    if negate:
        total = -total
    if c is not None:
        total += sum(grid(x, e0) for x in c)
    sign = -1 if total < 0 else 1
    rest = abs(total)
    limbs = []
    while rest and len(limbs) < p:
        lo = rest.bit_length() - 53
        chunk = rest >> lo if lo >= 0 else rest << -lo
        limbs.append(sign * float(Fraction(chunk) * Fraction(2) ** (lo + e0)))
        rest -= chunk << lo if lo >= 0 else rest
    return limbs + [0.0] * (p - len(limbs))


def call(L, p, words, e0, negate, c):
    W = (C.c_int64 * GW[p])(*words)
    out = (C.c_double * p)()
    cp = (C.c_double * p)(*c) if c is not None else None
    assert L.words_host_to_md(p, GW[p], W, e0, int(negate), cp, out) == 0
    return list(out)


def md_value(rng, p, top):
    """A normalised md value near 2^top with random lower limbs."""
    x = [rng.uniform(-1, 1) * 2.0 ** top]
    for _ in range(p - 1):
        x.append(x[-1] * 2.0 ** -53 * rng.uniform(-1, 1))
    return x


@pytest.mark.parametrize("p", [2, 4, 8])
def test_words_to_md_matches_exact_greedy_truncation(lib, p):
    rng = random.Random(7 + p)
    gw = GW[p]
    for trial in range(600):
        kind = trial % 6
        if kind == 0:    # random words of both signs near the bound
            words = [rng.randint(-2 ** 56, 2 ** 56) for _ in range(gw - 3)] + [0, 0, 0]
        elif kind == 1:  # carries across every boundary
            words = [rng.choice([2 ** 32 - 1, -1, 2 ** 33, -(2 ** 33)]) for _ in range(gw - 3)] + [0, 0, 0]
        elif kind == 2:  # long zero runs between the significant bits
            words = [0] * gw
            for g in rng.sample(range(gw - 3), 3):
                words[g] = rng.choice([1, -1]) << rng.randint(0, 40)
        elif kind == 3:  # exact cancellation to zero
            words = [0] * gw
            words[1] = 2 ** 40
            words[2] = -(2 ** 8)
        else:
            words = [rng.randint(-2 ** 40, 2 ** 40) for _ in range(gw - 3)] + [0, 0, 0]
        e0 = rng.randint(-700, 100)
        negate = rng.random() < 0.5
        c = None
        if kind >= 4:
            # md addends below, inside and above the range of the words
            top = e0 + rng.randint(-80, 32 * (gw - 3) + 20)
            c = md_value(rng, p, top)
        got = call(lib, p, words, e0, negate, c)
        want = expected(p, words, e0, negate, c)
        assert got == want, (p, trial, kind, got, want)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_words_to_md_limbs_are_normalised(lib, p):
    rng = random.Random(100 + p)
    for _ in range(200):
        words = [rng.randint(-2 ** 56, 2 ** 56) for _ in range(GW[p] - 3)] + [0, 0, 0]
        out = call(lib, p, words, rng.randint(-500, 0), False, None)
        for a, b in zip(out, out[1:]):
            if b != 0.0:
                assert abs(b) < np.spacing(abs(a)) and np.sign(a) == np.sign(b)
