"""Pins of the complex oracle (Hermitian Householder QR, back substitution and
least squares on complex multiple doubles, the paper's Section 3 remark on
complex data) against exact Gaussian-rational arithmetic (pairs of
fractions.Fraction) on small systems:

* least squares equals the exact solution of the normal equations
  A^H A x = A^H b to within 2^(12 - 53p) of its size;
* QR: A = Q R and Q^H Q = I to within 2^(12 - 53p), R upper triangular with
  exact zeros below, and R^H R = A^H A (R's diagonal carries the phases of
  the reflected columns' leading entries);
* back substitution equals exact elimination;
* special cases: real data give the real oracle's solution with exactly zero
  imaginary parts; data times i give the solution times -i.
A dropped conjugation or a wrong reflector phase fails the first two."""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle

PRECS = [2, 4, 8]


def cz(re, im):
    return (Fraction(re), Fraction(im))


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cconj(a):
    return (a[0], -a[1])


def cdiv(a, b):
    d = b[0] * b[0] + b[1] * b[1]
    n = cmul(a, cconj(b))
    return (n[0] / d, n[1] / d)


def czero():
    return (Fraction(0), Fraction(0))


def csum(it):
    acc = czero()
    for v in it:
        acc = cadd(acc, v)
    return acc


def csolve(M, rhs):
    n = len(M)
    a = [list(M[i]) + [rhs[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if a[r][c] != czero())
        a[c], a[piv] = a[piv], a[c]
        for r in range(n):
            if r != c and a[r][c] != czero():
                f = cdiv(a[r][c], a[c][c])
                a[r] = [csub(x, cmul(f, y)) for x, y in zip(a[r], a[c])]
    return [cdiv(a[i][n], a[i][i]) for i in range(n)]


def to_planar(p, M):
    """list-of-rows of complex Fractions (dyadic) -> (re, im) limb-planar (p, n, m)"""
    m, n = len(M), len(M[0])
    re, im = np.zeros((p, n, m)), np.zeros((p, n, m))
    for i in range(m):
        for j in range(n):
            re[0, j, i] = float(M[i][j][0])
            im[0, j, i] = float(M[i][j][1])
    return re, im


def from_planar(re, im):
    p, n, m = re.shape
    return [[(sum((Fraction(float(re[l, j, i])) for l in range(p)), Fraction(0)),
              sum((Fraction(float(im[l, j, i])) for l in range(p)), Fraction(0))) for j in range(n)]
            for i in range(m)]


def vec(re, im):
    p, n = re.shape
    return [(sum((Fraction(float(re[l, i])) for l in range(p)), Fraction(0)),
             sum((Fraction(float(im[l, i])) for l in range(p)), Fraction(0))) for i in range(n)]


def rand_cmatrix(rng, m, n, lo=-9, hi=9):
    return [[cz(rng.randint(lo, hi), rng.randint(lo, hi)) for _ in range(n)] for _ in range(m)]


def cabs(a):
    return abs(a[0]) + abs(a[1])


def close(got, ref, p, scale):
    return cabs(csub(got, ref)) <= scale * Fraction(2) ** (12 - 53 * p)


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("shape", [(4, 3), (6, 4), (7, 7)])
def test_zlstsq_exact_normal_equations(p, shape):
    rng = random.Random(100 * p + shape[0])
    m, n = shape
    A = rand_cmatrix(rng, m, n)
    b = [cz(rng.randint(-9, 9), rng.randint(-9, 9)) for _ in range(m)]
    AhA = [[csum(cmul(cconj(A[k][i]), A[k][j]) for k in range(m)) for j in range(n)] for i in range(n)]
    Ahb = [csum(cmul(cconj(A[k][i]), b[k]) for k in range(m)) for i in range(n)]
    xe = csolve(AhA, Ahb)
    Ar, Ai = to_planar(p, A)
    br = np.zeros((p, m)); bi = np.zeros((p, m))
    br[0] = [float(v[0]) for v in b]; bi[0] = [float(v[1]) for v in b]
    xr, xi = oracle.zlstsq(Ar, Ai, br, bi)
    got = vec(xr, xi)
    scale = max(cabs(v) for v in xe) * 100
    for g, e in zip(got, xe):
        assert close(g, e, p, scale)


@pytest.mark.parametrize("p", PRECS)
@pytest.mark.parametrize("shape", [(3, 3), (5, 3), (6, 6)])
def test_zqr_invariants(p, shape):
    rng = random.Random(7 * p + shape[0])
    m, n = shape
    A = rand_cmatrix(rng, m, n)
    Ar, Ai = to_planar(p, A)
    Rr, Ri, Qr, Qi, beta = oracle.zqr(Ar, Ai)
    R = from_planar(Rr, Ri)
    Q = from_planar(Qr, Qi)
    scale = max(cabs(v) for row in A for v in row) * 100
    for i in range(m):
        for j in range(n):
            if i > j:
                assert R[i][j] == czero()
            qr = csum(cmul(Q[i][k], R[k][j]) for k in range(m))
            assert close(qr, A[i][j], p, scale)
    for i in range(m):
        for j in range(m):
            g = csum(cmul(cconj(Q[k][i]), Q[k][j]) for k in range(m))
            assert close(g, cz(1 if i == j else 0, 0), p, 100)
    # R^H R = A^H A (the Cholesky factor up to the phases of R's diagonal)
    for i in range(n):
        for j in range(n):
            rr = csum(cmul(cconj(R[k][i]), R[k][j]) for k in range(m))
            aa = csum(cmul(cconj(A[k][i]), A[k][j]) for k in range(m))
            assert close(rr, aa, p, scale * scale)


@pytest.mark.parametrize("p", PRECS)
def test_zqr_diagonal_phase_convention(p):
    """The first column x reflects to e^{i arg x0} ||x|| e1."""
    A = [[cz(3, 4)], [cz(0, 12)], [cz(0, 0)]]      # ||x|| = 13, x0 / |x0| = (3 + 4i) / 5
    Ar, Ai = to_planar(p, A)
    Rr, Ri, _, _, _ = oracle.zqr(Ar, Ai, want_q=False)
    r00 = (sum(Fraction(float(v)) for v in Rr[:, 0, 0]), sum(Fraction(float(v)) for v in Ri[:, 0, 0]))
    assert close(r00, (Fraction(39, 5), Fraction(52, 5)), p, 100)


@pytest.mark.parametrize("p", PRECS)
def test_zbacksub_exact(p):
    rng = random.Random(11 + p)
    n = 7
    R = [[(cz(rng.randint(1, 5), rng.randint(-5, 5)) if i == j else
           (cz(rng.randint(-9, 9), rng.randint(-9, 9)) if j > i else czero())) for j in range(n)] for i in range(n)]
    y = [cz(rng.randint(-9, 9), rng.randint(-9, 9)) for _ in range(n)]
    x = [czero()] * n
    for i in reversed(range(n)):
        s = y[i]
        for j in range(i + 1, n):
            s = csub(s, cmul(R[i][j], x[j]))
        x[i] = cdiv(s, R[i][i])
    Rr, Ri = to_planar(p, R)
    yr = np.zeros((p, n)); yi = np.zeros((p, n))
    yr[0] = [float(v[0]) for v in y]; yi[0] = [float(v[1]) for v in y]
    xr, xi = oracle.zbacksub(Rr, Ri, yr, yi)
    scale = max(cabs(v) for v in x) * 100
    for g, e in zip(vec(xr, xi), x):
        assert close(g, e, p, scale)


@pytest.mark.parametrize("p", PRECS)
def test_real_data_and_times_i(p):
    import synth
    m, n = 30, 20
    A, b = synth.lstsq_problem(p, m, n, seed=4, tag="zreal")
    z = np.zeros_like(A)
    zb = np.zeros_like(b)
    xr, xi = oracle.zlstsq(A, z, b, zb)
    x = oracle.lstsq(A, b)
    assert np.all(xi == 0.0)
    assert oracle.rel_err(xr, x) < 2.0 ** (20 - 53 * p)
    # i A x = i b has the same solution; A (i x) = b gives x times -i
    xr2, xi2 = oracle.zlstsq(z, A, b, zb)
    assert oracle.rel_err(xi2, -x) < 2.0 ** (20 - 53 * p)
    assert np.max(np.abs(xr2[0])) <= 2.0 ** (20 - 53 * p) * np.max(np.abs(x[0]))
