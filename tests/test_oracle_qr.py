"""Pins of the oracle's Householder QR, back substitution and least squares.

Reference points that do not come from the oracle itself: exact rational
arithmetic (``fractions.Fraction``) on small integer systems, the invariants
of a QR factorisation (Q^T Q = I, A = QR, R^T R = A^T A, positive diagonal),
closed-form special cases, and closed-form operation counts.  The method:
arXiv 2110.08375, Section 1 (A = QR reduces Ax = b to Rx = Q^T b), Section 3
(Householder reflectors with the sign convention of Golub & Van Loan,
Algorithm 5.1.1, so that P x = ||x|| e1), Section 2 (back substitution).
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle

PRECS = [2, 4, 8]


def md_from_int(p, M):
    """integer (or dyadic) matrix given as list of rows -> limb-planar (p, n, m)"""
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    out = np.zeros((p, n, m))
    out[0] = M.T
    return out


def to_frac(X):
    """limb-planar (p, cols, rows) -> rows x cols Fraction matrix"""
    p, cols, rows = X.shape
    return [[sum((Fraction(float(X[l, j, i])) for l in range(p)), Fraction(0))
             for j in range(cols)] for i in range(rows)]


def vec_frac(x):
    p, n = x.shape
    return [sum((Fraction(float(x[l, i])) for l in range(p)), Fraction(0)) for i in range(n)]


def matmul(A, B):
    return [[sum((A[i][k] * B[k][j] for k in range(len(B))), Fraction(0))
             for j in range(len(B[0]))] for i in range(len(A))]


def transpose(A):
    return [list(r) for r in zip(*A)]


def solve(M, rhs):
    """exact Gaussian elimination"""
    n = len(M)
    a = [list(M[i]) + [rhs[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[piv] = a[piv], a[c]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c] / a[c][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [a[i][n] / a[i][i] for i in range(n)]


def maxabs(A):
    return max(abs(x) for row in A for x in row)


def rand_int_matrix(rng, m, n, lo=-9, hi=9):
    while True:
        M = [[rng.randint(lo, hi) for _ in range(n)] for _ in range(m)]
        if np.linalg.matrix_rank(np.array(M, dtype=float)) == n and \
                np.linalg.cond(np.array(M, dtype=float)) < 200:
            return M


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("shape", [(4, 4), (6, 3), (8, 5), (5, 1), (7, 6)])
def test_qr_invariants_exact(p, shape):
    m, n = shape
    rng = random.Random(100 * p + 10 * m + n)
    Aint = rand_int_matrix(rng, m, n)
    A = md_from_int(p, Aint)
    R, Q, beta = oracle.qr(A)
    Rf, Qf, Af = to_frac(R), to_frac(Q), [[Fraction(v) for v in r] for r in Aint]
    u = Fraction(2) ** (-53 * p)
    tol = 1000 * m * n * u
    # R upper triangular with exactly zero entries below the diagonal, positive diagonal
    for i in range(m):
        for j in range(n):
            if i > j:
                assert Rf[i][j] == 0
        if i < n:
            assert Rf[i][i] > 0
    nA = maxabs(Af)
    # A = QR
    QR = matmul(Qf, Rf)
    assert maxabs([[QR[i][j] - Af[i][j] for j in range(n)] for i in range(m)]) <= tol * nA
    # Q^T Q = I
    QtQ = matmul(transpose(Qf), Qf)
    assert maxabs([[QtQ[i][j] - (1 if i == j else 0) for j in range(m)] for i in range(m)]) <= tol
    # R^T R = A^T A  (R is the Cholesky factor of A^T A, unique with positive diagonal)
    RtR = matmul(transpose(Rf[:n]), Rf[:n])
    AtA = matmul(transpose(Af), Af)
    assert maxabs([[RtR[i][j] - AtA[i][j] for j in range(n)] for i in range(n)]) <= tol * nA * nA


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("shape", [(5, 5), (7, 4), (9, 6), (3, 1)])
def test_lstsq_exact_normal_equations(p, shape):
    m, n = shape
    rng = random.Random(7 * p + m * n)
    Aint = rand_int_matrix(rng, m, n)
    bint = [rng.randint(-9, 9) for _ in range(m)]
    A = md_from_int(p, Aint)
    b = np.zeros((p, m)); b[0] = bint
    x = oracle.lstsq(A, b)
    Af = [[Fraction(v) for v in r] for r in Aint]
    At = transpose(Af)
    xstar = solve(matmul(At, Af), [sum(At[i][k] * bint[k] for k in range(m)) for i in range(n)])
    xf = vec_frac(x)
    cond = np.linalg.cond(np.array(Aint, dtype=float))
    tol = Fraction(2) ** (-53 * p) * Fraction(int(1000 * m * n * cond * cond) + 1)
    nx = max(abs(v) for v in xstar)
    assert max(abs(a - b) for a, b in zip(xf, xstar)) <= tol * max(nx, 1)


@pytest.mark.parametrize("p", PRECS)
def test_lstsq_consistent_recovers_dyadic_solution(p):
    rng = random.Random(55 + p)
    m, n = 9, 6
    Aint = rand_int_matrix(rng, m, n)
    xstar = [Fraction(rng.randint(-64, 64), 8) for _ in range(n)]
    bint = [sum(Aint[i][k] * xstar[k] for k in range(n)) for i in range(m)]
    A = md_from_int(p, Aint)
    b = np.zeros((p, m)); b[0] = [float(v) for v in bint]
    xf = vec_frac(oracle.lstsq(A, b))
    cond = np.linalg.cond(np.array(Aint, dtype=float))
    tol = Fraction(2) ** (-53 * p) * Fraction(int(1000 * n * cond) + 1)
    assert max(abs(a - b) for a, b in zip(xf, xstar)) <= tol * 8


@pytest.mark.parametrize("p", PRECS)
def test_single_column(p):
    a = [3, -1, 2, 5]
    bb = [1, 2, -4, 7]
    A = md_from_int(p, [[v] for v in a])
    b = np.zeros((p, 4)); b[0] = bb
    x = vec_frac(oracle.lstsq(A, b))[0]
    exact = Fraction(sum(u * v for u, v in zip(a, bb)), sum(u * u for u in a))
    assert abs(x - exact) <= Fraction(2) ** (4 - 53 * p) * abs(exact)


@pytest.mark.parametrize("p", PRECS)
def test_diagonal_and_triangular_are_exact(p):
    D = [[-3, 0, 0], [0, 2, 0], [0, 0, -0.5]]
    R, Q, _ = oracle.qr(md_from_int(p, D))
    assert to_frac(R) == [[3, 0, 0], [0, 2, 0], [0, 0, Fraction(1, 2)]]
    assert to_frac(Q) == [[-1, 0, 0], [0, 1, 0], [0, 0, -1]]
    U = [[2, 1, -1], [0, 3, 4], [0, 0, 5], [0, 0, 0]]
    R, Q, _ = oracle.qr(md_from_int(p, U))
    assert to_frac(R) == [[Fraction(v) for v in r] for r in U]
    assert to_frac(Q) == [[1 if i == j else 0 for j in range(4)] for i in range(4)]


@pytest.mark.parametrize("p", PRECS)
def test_orthogonal_input_gives_identity_R(p):
    H = [[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]]
    A = [[v / 2 for v in r] for r in H]          # orthogonal, dyadic
    R, Q, _ = oracle.qr(md_from_int(p, A))
    tol = Fraction(2) ** (8 - 53 * p)
    Rf, Qf = to_frac(R), to_frac(Q)
    for i in range(4):
        for j in range(4):
            assert abs(Rf[i][j] - (1 if i == j else 0)) <= tol
            assert abs(Qf[i][j] - Fraction(A[i][j])) <= tol


@pytest.mark.parametrize("p", PRECS)
def test_backsub_exact(p):
    rng = random.Random(300 + p)
    n = 12
    U = [[0] * n for _ in range(n)]
    for i in range(n):
        U[i][i] = rng.randint(1, 9) * rng.choice([-1, 1])
        for j in range(i + 1, n):
            U[i][j] = rng.randint(-9, 9)
    y = [rng.randint(-9, 9) for _ in range(n)]
    R = md_from_int(p, U)
    yy = np.zeros((p, n)); yy[0] = y
    x = vec_frac(oracle.backsub(R, yy))
    xstar = solve([[Fraction(v) for v in r] for r in U], [Fraction(v) for v in y])
    cond = np.linalg.cond(np.array(U, dtype=float))
    tol = Fraction(2) ** (-53 * p) * Fraction(int(100 * n * cond) + 1)
    nx = max(abs(v) for v in xstar)
    assert max(abs(a - b) for a, b in zip(x, xstar)) <= tol * nx


@pytest.mark.parametrize("p", PRECS)
def test_backsub_tiled_identity_3x3(p):
    """Algorithm 1 on the paper's 3-by-3 tiled example (Section 2): with the
    diagonal tiles inverted, x3 = U3^{-1} b3, b2 -= A23 x3, b1 -= A13 x3,
    x2 = U2^{-1} b2, b1 -= A12 x2, x1 = U1^{-1} b1 gives the same x as the
    plain row-by-row solve.  Checked in exact rationals against the oracle."""
    rng = random.Random(400 + p)
    t, N = 2, 3
    n = t * N
    U = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        U[i][i] = Fraction(rng.randint(1, 5))
        for j in range(i + 1, n):
            U[i][j] = Fraction(rng.randint(-3, 3))
    b = [Fraction(rng.randint(-5, 5)) for _ in range(n)]

    def blk(i, j):
        return [r[j * t:(j + 1) * t] for r in U[i * t:(i + 1) * t]]

    def inv_upper(T):
        k = len(T)
        cols = [solve(T, [Fraction(int(r == c)) for r in range(k)]) for c in range(k)]
        return transpose(cols)

    def mv(M, v):
        return [sum((M[i][k] * v[k] for k in range(len(v))), Fraction(0)) for i in range(len(M))]

    bb = [b[i * t:(i + 1) * t] for i in range(N)]
    x = [None] * N
    for i in range(N - 1, -1, -1):
        x[i] = mv(inv_upper(blk(i, i)), bb[i])
        for j in range(i):
            upd = mv(blk(j, i), x[i])
            bb[j] = [u - v for u, v in zip(bb[j], upd)]
    xt = [v for blk_ in x for v in blk_]
    assert xt == solve(U, b)
    R = md_from_int(p, [[float(v) for v in r] for r in U])
    yy = np.zeros((p, n)); yy[0] = [float(v) for v in b]
    xo = vec_frac(oracle.backsub(R, yy))
    assert max(abs(a - c) for a, c in zip(xo, xt)) <= Fraction(2) ** (10 - 53 * p) * max(map(abs, xt))


@pytest.mark.parametrize("p", [2, 4])
def test_rank_deficient_reports_zero_pivot(p):
    A = md_from_int(p, [[1, 0], [2, 0], [3, 0]])
    b = np.zeros((p, 3)); b[0] = [1, 2, 3]
    with pytest.raises(ZeroDivisionError):
        oracle.lstsq(A, b)


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("shape", [(7, 4), (5, 5), (9, 3)])
def test_operation_counts_closed_form(p, shape):
    m, n = shape
    rng = random.Random(900 + m + n + p)
    Aint = rand_int_matrix(rng, m, n)
    A = md_from_int(p, Aint)
    for want_q in (False, True):
        oracle.reset_counts()
        oracle.qr(A, want_q=want_q)
        got = oracle.counts()
        degenerate = {n - 1} if m == n else set()
        ident = set()
        if m == n:
            # the last reflector of a square matrix is the identity iff the
            # last pivot came out >= 0; the oracle tallies which branch it took
            if got["ident"]:
                ident = {n - 1}
        exp = oracle.qr_counts_closed_form(m, n, want_q, npos=got["pos_branch"],
                                           degenerate=degenerate, ident=ident)
        assert {k: got[k] for k in exp} == exp
        assert got["ident"] + got["flip"] == len(degenerate)
    # the x0 > 0 branch is taken exactly when the column's leading entry is > 0;
    # the first column is untouched by earlier reflectors
    oracle.reset_counts()
    B = [row[:] for row in Aint]
    for r in B:
        r[0] = abs(r[0]) + 1
    oracle.qr(md_from_int(p, [r[:1] for r in B]), want_q=False)
    assert oracle.counts()["pos_branch"] == 1
    # least squares = QR applied to b, then back substitution
    b = np.zeros((p, m)); b[0] = [rng.randint(-5, 5) for _ in range(m)]
    oracle.reset_counts()
    oracle.lstsq(A, b)
    got = oracle.counts()
    degenerate = {n - 1} if m == n else set()
    ident = {n - 1} if (m == n and got["ident"]) else set()
    exp = oracle.qr_counts_closed_form(m, n, False, npos=got["pos_branch"], degenerate=degenerate,
                                       ident=ident, extra_cols=1)
    bs = oracle.backsub_counts_closed_form(n)
    for k in exp:
        exp[k] += bs[k]
    assert {k: got[k] for k in exp} == exp


@pytest.mark.parametrize("p", PRECS)
def test_gemm_gemv_exact_small(p):
    rng = random.Random(77 + p)
    A = [[rng.randint(-9, 9) for _ in range(3)] for _ in range(4)]
    B = [[rng.randint(-9, 9) for _ in range(2)] for _ in range(3)]
    Cm = oracle.gemm(md_from_int(p, A), md_from_int(p, B))
    assert to_frac(Cm) == matmul([[Fraction(v) for v in r] for r in A],
                                 [[Fraction(v) for v in r] for r in B])
    x = np.zeros((p, 3)); x[0] = [1, -2, 3]
    y = oracle.gemv(md_from_int(p, A), x)
    assert vec_frac(y) == [sum(A[i][k] * [1, -2, 3][k] for k in range(3)) for i in range(4)]
    z = np.zeros((p, 4)); z[0] = [1, 0, -1, 2]
    yt = oracle.gemv(md_from_int(p, A), z, trans=True)
    assert vec_frac(yt) == [sum(A[i][k] * [1, 0, -1, 2][i] for i in range(4)) for k in range(3)]


@pytest.mark.parametrize("p", PRECS)
def test_random_md_inputs_against_float_qr(p):
    """Full md inputs from the seeded generator: R matches numpy's double QR
    (after sign normalisation) to double accuracy, and A = QR holds to md
    accuracy when evaluated with the oracle's own exact differences."""
    import synth
    m, n = 12, 7
    A, b = synth.lstsq_problem(p, m, n, seed=3)
    R, Q, _ = oracle.qr(A)
    Ad = A[0].T
    _, Rn = np.linalg.qr(Ad)
    Rn = Rn * np.sign(np.diag(Rn))[:, None]
    assert np.allclose(R[0].T[:n], Rn, atol=1e-13)
    QR = oracle.gemm(Q, R)
    assert oracle.rel_err(QR, A) < 2.0 ** (-53 * p) * 1e4
