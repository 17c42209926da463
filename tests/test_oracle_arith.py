"""Pins of the oracle's multiple-double arithmetic against exact arithmetic.

The oracle defines each md operation as the exact result rounded to p limbs
(arXiv 2110.08375, Section 1.1: a multiple double is an unevaluated sum of
doubles).  These tests check it against Python's exact rationals
(``fractions.Fraction``) and 450-digit decimals, so a dropped partial product,
a lost carry, a wrong sign or a wrong limb order fails here.
"""
import math
import os
import random
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
PRECS = [2, 4, 8]


def F(limbs) -> Fraction:
    return sum((Fraction(float(x)) for x in np.ravel(limbs)), Fraction(0))


def rnd_md(rng: random.Random, p: int, scale_exp: int = 0) -> np.ndarray:
    """A normalised md number with random limbs (each under half an ulp of the
    one above), top limb of magnitude about 2**scale_exp."""
    x = np.zeros(p)
    x[0] = rng.uniform(-1, 1) * 2.0 ** scale_exp
    for i in range(1, p):
        x[i] = x[i - 1] * 2.0 ** -54 * rng.uniform(-1, 1)
    return x


def is_normalized(c: np.ndarray) -> bool:
    for i in range(len(c) - 1):
        if c[i] == 0.0:
            if np.any(c[i + 1:] != 0.0):
                return False
            return True
        if abs(c[i + 1]) > math.ulp(c[i]) / 2:
            return False
    return True


def test_two_sum_exact():
    rng = random.Random(1)
    cases = [(1.0, 2.0 ** -60), (1e300, -1e300), (0.1, 0.2), (2.0 ** 52, 0.5), (-3.5, 3.5)]
    for _ in range(20000):
        e1, e2 = rng.randint(-200, 200), rng.randint(-200, 200)
        cases.append((rng.uniform(-1, 1) * 2.0 ** e1, rng.uniform(-1, 1) * 2.0 ** e2))
    for a, b in cases:
        s, e = oracle.two_sum(a, b)
        assert Fraction(s) + Fraction(e) == Fraction(a) + Fraction(b)
        assert s == a + b
        assert abs(e) <= math.ulp(s) / 2 or s == 0


def test_two_prod_exact():
    rng = random.Random(2)
    cases = [(1.0 + 2.0 ** -52, 1.0 + 2.0 ** -52), (3.0, 1.0 / 3.0), (0.1, 0.1)]
    for _ in range(20000):
        e1, e2 = rng.randint(-300, 300), rng.randint(-300, 300)
        cases.append((rng.uniform(-1, 1) * 2.0 ** e1, rng.uniform(-1, 1) * 2.0 ** e2))
    for a, b in cases:
        p, e = oracle.two_prod(a, b)
        assert Fraction(p) + Fraction(e) == Fraction(a) * Fraction(b)


@pytest.mark.parametrize("p", PRECS)
def test_add_sub_mul_exact_rounding(p):
    """|c - exact| <= 2^(1-53p) |exact| and the limbs are normalised."""
    rng = random.Random(10 + p)
    tol = Fraction(2) ** (1 - 53 * p)
    for t in range(600):
        a = rnd_md(rng, p, rng.randint(-30, 30))
        if t % 5 == 0:       # heavy cancellation: b = -a + tiny
            b = -a.copy()
            b[p - 1] += math.ulp(a[p - 1]) * rng.randint(-3, 3) if a[p - 1] else 0.0
            b[-1] = b[-1] + rnd_md(rng, 1, -60 * p)[0]
        elif t % 5 == 1:     # very different magnitudes
            b = rnd_md(rng, p, rng.randint(-300, -100))
        else:
            b = rnd_md(rng, p, rng.randint(-30, 30))
        for op, exact in (("add", F(a) + F(b)), ("sub", F(a) - F(b)), ("mul", F(a) * F(b))):
            c = getattr(oracle, op)(a, b)
            assert is_normalized(c), (op, a, b, c)
            err = abs(F(c) - exact)
            assert err <= tol * abs(exact), (op, p, float(err / abs(exact)) if exact else err)


@pytest.mark.parametrize("p", PRECS)
def test_div_exact_rounding(p):
    rng = random.Random(20 + p)
    tol = Fraction(2) ** (2 - 53 * p)
    for t in range(300):
        a = rnd_md(rng, p, rng.randint(-40, 40))
        b = rnd_md(rng, p, rng.randint(-40, 40))
        if b[0] == 0:
            continue
        c = oracle.div(a, b)
        exact = F(a) / F(b)
        assert is_normalized(c)
        assert abs(F(c) - exact) <= tol * abs(exact)
    # exact quotients come out exact
    a = np.zeros(p); a[0] = 1.0
    b = np.zeros(p); b[0] = 4.0
    assert F(oracle.div(a, b)) == Fraction(1, 4)
    a[0] = 7.0; b[0] = 3.0
    q = oracle.div(a, b)
    assert abs(F(q) - Fraction(7, 3)) <= tol * Fraction(7, 3)


@pytest.mark.parametrize("p", PRECS)
def test_sqrt_against_decimal(p):
    getcontext().prec = 450
    rng = random.Random(30 + p)
    tol = Decimal(2) ** (3 - 53 * p)
    for _ in range(120):
        a = np.abs(rnd_md(rng, p, rng.randint(-60, 60)))
        if a[0] == 0:
            continue
        a[1:] *= np.sign(a[1:]) * np.sign(rng.uniform(-1, 1))   # signs of lower limbs random
        c = oracle.sqrt(a)
        exact = sum(Decimal(float(x)) for x in a).sqrt()
        got = sum(Decimal(float(x)) for x in c)
        assert abs(got - exact) <= tol * exact
        assert is_normalized(c)
    # perfect squares are exact
    a = np.zeros(p); a[0] = 9.0
    assert F(oracle.sqrt(a)) == 3
    assert F(oracle.sqrt(np.zeros(p))) == 0


@pytest.mark.parametrize("p", PRECS)
def test_normalize_and_diff(p):
    rng = random.Random(40 + p)
    for _ in range(200):
        raw = np.array([rng.uniform(-1, 1) * 2.0 ** (-40 * i) for i in range(p)])
        c = oracle.normalize(raw)
        assert is_normalized(c)
        assert abs(F(c) - F(raw)) <= Fraction(2) ** (1 - 53 * p) * abs(F(raw))
        a = rnd_md(rng, p)
        b = rnd_md(rng, p)
        d = oracle.diff(a[:, None], b[:, None])[0]
        assert d == float(F(a) - F(b))   # Fraction -> float rounds to nearest


def test_table1_fixture_consistent():
    """Table 1 of the paper (flop convention): each row's +,-,*,/ add up to its
    Sigma, the printed averages are the means of the Sigma column, and the
    oracle's multipliers are the fixture's."""
    rows, avgs = {}, {}
    with open(os.path.join(HERE, "golden", "table1_opcounts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "avg":
                avgs[line[1]] = float(line[2])
            else:
                rows[(line[0], line[1])] = tuple(int(v) for v in line[2:])
    pmap = {"dd": 2, "qd": 4, "od": 8}
    for (prec, op), vals in rows.items():
        assert sum(vals[:4]) == vals[4]
        assert oracle.TABLE1[pmap[prec]][op] == vals
    for prec, avg in avgs.items():
        s = [rows[(prec, op)][4] for op in ("add", "mul", "div")]
        assert round(sum(s) / 3, 1) == avg
    # the per-precision overhead factors of the paper's Section 4.3 (11.7, 5.4)
    assert round(avgs["qd"] / avgs["dd"], 1) == 11.7
    assert round(avgs["od"] / avgs["qd"], 1) == 5.4
