"""Closed-form least-squares solution of the precision-mode workload.

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

For A = U diag(sigma) V^T with U (m x n) orthonormal columns and V (n x n)
orthogonal, the least-squares solution of A x = b is
    x* = V diag(1/sigma) U^T b
(the pseudo-inverse of A applied to b; Section 1 states the problem as the
minimiser of ||b - A x||).  The workload's factors are Walsh-Hadamard based
(synth.modes_structure):
    U   = D_u H_m[:, c] / sqrt(m),
    V^T = H_n[pi, :] D_v / sqrt(n),
    sigma_k = D_k 2^-20 / sqrt(2),
so that
    x* = 2^(20 - (log2 n - 1)/2 - log2(m)/2) D_v H_n[:, pi] diag(1/D) H_m[c, :] D_u b.
This module evaluates that formula with Python integers: b exactly, the two
Walsh-Hadamard products exactly, the divisions by D_k to 1024 fractional
bits, and rounds the result to p doubles greedily (x0 = RN(x), x1 = RN(x - x0),
...), the oracle's rounding of an exact value.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

GUARD_BITS = 1024


def _hadamard_apply(v: list) -> list:
    """H_N v for Sylvester's H_N, H_N[i, j] = (-1)^popcount(i & j), straight
    from that definition's recursive form H_2N = [[H_N, H_N], [H_N, -H_N]]."""
    N = len(v)
    if N == 1:
        return list(v)
    top = _hadamard_apply(v[:N // 2])
    bot = _hadamard_apply(v[N // 2:])
    return [a + b for a, b in zip(top, bot)] + [a - b for a, b in zip(top, bot)]


def _exact(limbs) -> Fraction:
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))


def round_md(v: Fraction, p: int) -> list:
    """Greedy rounding of an exact rational to p doubles."""
    out = []
    r = v
    for _ in range(p):
        d = float(r)          # Fraction -> float rounds to nearest
        out.append(d)
        r = r - Fraction(d)
    return out


def modes_solution(st: dict, b: np.ndarray, p: int) -> np.ndarray:
    """x* = V diag(1/sigma) U^T b for the structure ``st`` of
    synth.modes_structure and b of shape (pb, m); returns (p, n)."""
    m, n = st["m"], st["n"]
    lm, ln = int(math.log2(m)), int(math.log2(n))
    bx = [_exact(b[:, i]) for i in range(m)]
    E = max(v.denominator.bit_length() - 1 for v in bx)           # denominators are powers of 2
    bnum = [int(v * (1 << E)) for v in bx]
    g = _hadamard_apply([int(st["du"][i]) * bnum[i] for i in range(m)])   # H_m D_u b
    z = [0] * n
    for k in range(n):
        num = g[int(st["c"][k])] << GUARD_BITS
        D = int(st["D"][k])
        q = (abs(num) + D // 2) // D                                   # |num| / D to the nearest integer
        z[int(st["pi"][k])] = q if num >= 0 else -q
    h = _hadamard_apply(z)                                             # H_n[:, pi] diag(1/D) ...
    shift = 20 - (ln - 1) // 2 - lm // 2 - E - GUARD_BITS
    x = np.zeros((p, n))
    for j in range(n):
        v = Fraction(int(st["dv"][j]) * h[j]) * (Fraction(2) ** shift)
        x[:, j] = round_md(v, p)
    return x
