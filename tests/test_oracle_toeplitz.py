"""Pins of the oracle's block-Toeplitz solve (oracle.toeplitz_lstsq: block
forward substitution J_0 x_k = b_k - sum_{i=1}^{k} J_i x_{k-i}, each block in
the least-squares sense):

* square integer blocks: equal to exact rational block forward substitution;
* square blocks: equal to the oracle's least squares of the assembled
  (d+1) n x (d+1) n block lower triangular matrix (one QR of the whole
  system: another route to the same unique solution);
* tall blocks, consistent right-hand side b(t) = J(t) x*(t) mod t^{d+1}
  formed exactly: x* recovered."""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from test_oracle_qr import solve

PRECS = [2, 4, 8]


def blocks_int(rng, d1, m, n, p, diag_boost=0):
    J = np.zeros((p, d1, n, m))
    Jf = []
    for i in range(d1):
        M = [[Fraction(rng.randint(-9, 9) + (diag_boost if (i == 0 and r == c) else 0)) for c in range(n)]
             for r in range(m)]
        Jf.append(M)
        for r in range(m):
            for c in range(n):
                J[0, i, c, r] = float(M[r][c])
    return J, Jf


@pytest.mark.parametrize("p", PRECS)
def test_square_blocks_exact(p):
    rng = random.Random(5 + p)
    d1, n = 3, 3
    J, Jf = blocks_int(rng, d1, n, n, p, diag_boost=20)
    bf = [[Fraction(rng.randint(-9, 9)) for _ in range(n)] for _ in range(d1)]
    b = np.zeros((p, d1, n))
    for k in range(d1):
        b[0, k] = [float(v) for v in bf[k]]
    xf = []
    for k in range(d1):
        r = list(bf[k])
        for i in range(1, k + 1):
            r = [r[row] - sum(Jf[i][row][c] * xf[k - i][c] for c in range(n)) for row in range(n)]
        xf.append(solve(Jf[0], r))
    x = oracle.toeplitz_lstsq(J, b)
    for k in range(d1):
        for c in range(n):
            got = sum(Fraction(float(v)) for v in x[:, k, c])
            assert abs(got - xf[k][c]) <= (abs(xf[k][c]) + 1) * Fraction(2) ** (12 - 53 * p)


@pytest.mark.parametrize("p", PRECS)
def test_square_blocks_equal_the_assembled_system(p):
    import synth
    d1, n = 4, 6
    J = np.stack([synth.md_matrix(p, n, n, 3, f"toe/J{i}") for i in range(d1)], axis=1)
    J[0, 0] += 4.0 * np.eye(n)            # a well-conditioned diagonal block
    b = np.stack([synth.md_vector(p, n, 3, f"toe/b{k}") for k in range(d1)], axis=1)
    x = oracle.toeplitz_lstsq(J, b)
    N = d1 * n
    big = np.zeros((p, N, N))              # (p, cols, rows)
    for k in range(d1):
        for i in range(k + 1):
            big[:, (k - i) * n:(k - i + 1) * n, k * n:(k + 1) * n] = J[:, i]
    xb = oracle.lstsq(big, b.reshape(p, N))
    assert oracle.rel_err(x.reshape(p, N), xb) < 2.0 ** (24 - 53 * p)


@pytest.mark.parametrize("p", PRECS)
def test_tall_consistent_recovers_solution(p):
    rng = random.Random(9 + p)
    d1, m, n = 4, 8, 5
    J, Jf = blocks_int(rng, d1, m, n, p)
    xs = [[Fraction(rng.randint(-64, 64), 16) for _ in range(n)] for _ in range(d1)]
    b = np.zeros((p, d1, m))
    for k in range(d1):
        for r in range(m):
            v = sum(Jf[i][r][c] * xs[k - i][c] for i in range(k + 1) for c in range(n))
            b[0, k, r] = float(v)           # small integers over 16: exact doubles
    x = oracle.toeplitz_lstsq(J, b)
    for k in range(d1):
        for c in range(n):
            got = sum(Fraction(float(v)) for v in x[:, k, c])
            assert abs(got - xs[k][c]) <= 64 * Fraction(2) ** (20 - 53 * p)
