"""Pins of the precision-mode workload and its closed-form solution
(oracle/closed_form.py) against exact rational arithmetic.

* the generated A is exactly U diag(sigma) V^T with U^T U = I and V^T V = I
  (integer matrices, no rounding anywhere);
* the closed form V diag(1/sigma) U^T b equals the exact solution of the
  normal equations A^T A x = A^T b (Fraction Gaussian elimination), rounded
  to p doubles, for inconsistent right-hand sides;
* on consistent systems (b = A x*) it returns x* exactly, and b = A x* holds
  exactly in rationals;
* it agrees with the oracle's unblocked Householder least squares to
  kappa * n * u_p.
A wrong scale exponent, permutation, subset or sign in either the generator
or the closed form fails the first two."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import closed_form as cf
from test_oracle_qr import matmul, solve, to_frac, transpose, vec_frac


def _dense_factors(st):
    m, n = st["m"], st["n"]
    Hm = synth.hadamard_rows(np.arange(m, dtype=np.int64), m)
    Hn = synth.hadamard_rows(np.arange(n, dtype=np.int64), n)
    U = st["du"][:, None] * Hm[:, st["c"]]            # sqrt(m) U
    Vt = Hn[st["pi"], :] * st["dv"][None, :]           # sqrt(n) V^T
    return U, Vt


@pytest.mark.parametrize("m,n", [(16, 8), (64, 32), (256, 128)])
def test_generator_factors_are_exactly_orthogonal(m, n):
    st = synth.modes_structure(m, n, 1e3, seed=1)
    U, Vt = _dense_factors(st)
    assert np.array_equal(U.T @ U, m * np.eye(n, dtype=np.int64))
    assert np.array_equal(Vt @ Vt.T, n * np.eye(n, dtype=np.int64))
    assert np.array_equal(U @ np.diag(st["D"]) @ Vt, synth.modes_matrix_int(st))
    # singular values d_k / sqrt(2) with d = D 2^-20: kappa as asked
    A = synth.modes_problem(2, m, n, 1e3, seed=1)["A"]
    s = np.linalg.svd(A[0].T, compute_uv=False)
    assert abs(s.max() / s.min() / 1e3 - 1) < 1e-9
    assert abs(s.max() - st["D"].max() * 2.0 ** -20 / math.sqrt(2)) < 1e-9 * s.max()


@pytest.mark.parametrize("p", [2, 4, 8])
def test_closed_form_equals_exact_normal_equation_solution(p):
    m, n = 16, 8
    pr = synth.modes_problem(p, m, n, 10.0, seed=2, consistent=False)
    A, b = pr["A"], pr["b"]
    Af = to_frac(A)
    AtA = matmul(transpose(Af), Af)
    Atb = [sum((Af[i][j] * bi for i, bi in enumerate(vec_frac(b))), Fraction(0)) for j in range(n)]
    xe = solve(AtA, Atb)
    x = cf.modes_solution(pr["structure"], b, p)
    for j in range(n):
        got = sum((Fraction(float(v)) for v in x[:, j]), Fraction(0))
        assert abs(got - xe[j]) <= abs(xe[j]) * Fraction(2) ** (1 - 53 * p), j
        assert x[:, j].tolist() == cf.round_md(xe[j], p)


@pytest.mark.parametrize("p", [4, 8])
def test_consistent_system_is_exact_and_recovered(p):
    m, n = 64, 32
    pr = synth.modes_problem(p, m, n, 1e3, seed=3)
    A, b, xs = pr["A"], pr["b"], pr["xstar"]
    Af = to_frac(A)
    xf = vec_frac(xs)
    bf = vec_frac(b)
    for i in range(m):
        assert sum((Af[i][j] * xf[j] for j in range(n)), Fraction(0)) == bf[i]
    assert np.array_equal(cf.modes_solution(pr["structure"], b, p), xs)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_closed_form_agrees_with_unblocked_householder(p):
    m, n, kappa = 64, 32, 1e3
    pr = synth.modes_problem(p, m, n, kappa, seed=4, consistent=False)
    x = cf.modes_solution(pr["structure"], pr["b"], p)
    xo = oracle.lstsq(pr["A"], pr["b"])
    assert oracle.rel_err(xo, x) < kappa * kappa * n * 2.0 ** (-53 * p)
