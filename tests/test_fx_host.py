"""The integer-digit arithmetic of the Householder panel (csrc/fx.cuh)
compiled for the host and checked against exact rational arithmetic.

Every multiple double is an exact rational (the sum of its limbs), so each
operation is compared with the exact result of the same operation on the
same rationals: products, sums with cancellation, reciprocals and square
roots by Newton's method, the fixed-point column format, dot products and
norms accumulated by digit diagonals, and the reflector update a -= w u.
The bounds are the ones the panel relies on: a relative error of a few units
of 2^(-53P) for scalar results (the final rounding to P limbs dominates)
and an absolute error of a few units of the column's last digit for the
fixed-point vector operations."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OPS = {"id": 0, "mul": 1, "add": 2, "sub": 3, "recip": 4, "rsqrt": 5, "sqrt": 6, "half": 7, "x32": 8}
PS = [2, 4, 8]


@pytest.fixture(scope="module")
def fx():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = os.path.join(tempfile.mkdtemp(), "fx_host.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
                    "-o", out, os.path.join(ROOT, "tests", "harness", "fx_host.cu")], check=True)
    L = C.CDLL(out)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    L.fx_digits.argtypes = [C.c_int, C.c_int]
    L.fx_scalar.argtypes = [C.c_int, C.c_int, C.c_long, dp, dp, dp]
    L.fx_fixed_roundtrip.argtypes = [C.c_int, C.c_long, dp, C.c_int, dp, ip]
    L.fx_dot.argtypes = [C.c_int, C.c_int, C.c_long, dp, dp, C.c_int, C.c_int, dp]
    L.fx_axpy.argtypes = [C.c_int, C.c_long, dp, dp, dp, C.c_int, C.c_int]
    L.fx_axpy.restype = C.c_int
    L.fx_house.argtypes = [C.c_int, C.c_long, dp, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_int)]
    L.fx_house_md.argtypes = [C.c_int, C.c_long, dp, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_int)]
    L.fx_house_dd.argtypes = [C.c_long, dp, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_int)]
    L.fx_panel_replay.argtypes = [C.c_int, C.c_long, C.c_long, dp, dp]
    L.dp, L.ip = dp, ip
    return L


def draw(rng, p, n, lo=-20, hi=20):
    x = np.zeros((p, n))
    x[0] = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(lo, hi, n)
    for i in range(1, p):
        x[i] = x[i - 1] * 2.0 ** -54 * rng.uniform(-1, 1, n)
    return x


def exact(x, i):
    return sum(Fraction(float(v)) for v in x[:, i])


def scalar(fx, p, op, a, b=None):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(a if b is None else b)
    c = np.zeros_like(a)
    fx.fx_scalar(p, OPS[op], a.shape[1], a.ctypes.data_as(fx.dp), b.ctypes.data_as(fx.dp),
                 c.ctypes.data_as(fx.dp))
    return c


def rel(got, want, scale=None):
    scale = abs(want) if scale is None else scale
    if scale == 0:
        return 0.0 if got == want else float("inf")
    return float(abs(got - want) / scale)


def test_digit_counts(fx):
    # 53P bits plus 64 bits of guard and headroom, in 24-bit digits
    for p in PS:
        d = fx.fx_digits(p, 0)
        assert 24 * d >= 53 * p + 64 and 24 * (d - 1) < 53 * p + 64
        assert fx.fx_digits(p, 1) == d + 1


@pytest.mark.parametrize("p", PS)
def test_roundtrip_is_exact_to_p_limbs(fx, p):
    rng = np.random.default_rng(1)
    a = draw(rng, p, 200)
    a[:, :3] = 0.0
    a[0, 1] = 2.0 ** -1060          # subnormal range
    a[0, 2] = -3.0
    r = scalar(fx, p, "id", a)
    for i in range(a.shape[1]):
        assert rel(exact(r, i), exact(a, i)) <= 2.0 ** (-53 * p + 2), i
    # limbs decrease and do not overlap: |x_{k+1}| < ulp(x_k)
    for i in range(a.shape[1]):
        for k in range(p - 1):
            if r[k + 1, i] != 0:
                assert abs(r[k + 1, i]) < np.spacing(abs(r[k, i])), (i, k)


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("op", ["mul", "add", "sub"])
def test_arith_against_rationals(fx, p, op):
    rng = np.random.default_rng(2 + p)
    a, b = draw(rng, p, 150), draw(rng, p, 150)
    b[:, :20] = -a[:, :20]                              # exact cancellation
    b[:, 20:40] = a[:, 20:40]
    b[p - 1, 20:40] *= 1.5                              # cancellation down to the last limb
    r = scalar(fx, p, op, a, b)
    for i in range(a.shape[1]):
        x, y = exact(a, i), exact(b, i)
        want = {"mul": x * y, "add": x + y, "sub": x - y}[op]
        scale = abs(x * y) if op == "mul" else abs(x) + abs(y)
        assert rel(exact(r, i), want, scale) <= 2.0 ** (-53 * p + 3), (i, op)


@pytest.mark.parametrize("p", PS)
def test_reciprocal_and_square_roots(fx, p):
    rng = np.random.default_rng(7 + p)
    a = draw(rng, p, 80, lo=-60, hi=60)
    r = scalar(fx, p, "recip", a)
    for i in range(a.shape[1]):
        assert rel(exact(r, i), 1 / exact(a, i)) <= 2.0 ** (-53 * p + 3), i
    pos = a * np.sign(a[0])                             # the values' absolute values
    rs = scalar(fx, p, "rsqrt", pos)
    sq = scalar(fx, p, "sqrt", pos)
    for i in range(pos.shape[1]):
        x = exact(pos, i)
        y = exact(rs, i)
        assert abs(float(y * y * x - 1)) <= 2.0 ** (-53 * p + 4), i   # y = x^-1/2
        s = exact(sq, i)
        assert abs(float(s * s / x - 1)) <= 2.0 ** (-53 * p + 4), i   # s = x^1/2
        assert s > 0 and y > 0


@pytest.mark.parametrize("p", PS)
def test_power_of_two_shifts(fx, p):
    rng = np.random.default_rng(3)
    a = draw(rng, p, 50)
    h, x = scalar(fx, p, "half", a), scalar(fx, p, "x32", a)
    for i in range(a.shape[1]):
        assert rel(exact(h, i), exact(a, i) / 2) <= 2.0 ** (-53 * p + 2)
        assert rel(exact(x, i), exact(a, i) * 32) <= 2.0 ** (-53 * p + 2)


def fixed(fx, p, x, e):
    x = np.ascontiguousarray(x)
    d = fx.fx_digits(p, 0)
    y = np.zeros_like(x)
    dig = np.zeros((d, x.shape[1]), dtype=np.int32)
    fx.fx_fixed_roundtrip(p, x.shape[1], x.ctypes.data_as(fx.dp), e, y.ctypes.data_as(fx.dp),
                          dig.ctypes.data_as(fx.ip))
    return y, dig


@pytest.mark.parametrize("p", PS)
def test_fixed_point_column_format(fx, p):
    """Digits are sign-consistent and below 2^24, their value is the entry
    truncated toward zero at the column's last digit 2^(24e)."""
    rng = np.random.default_rng(4)
    d = fx.fx_digits(p, 0)
    a = draw(rng, p, 120, lo=-30, hi=3)
    e = -(d - 1)                                        # |a| < 2^(24(e+D)-3) = 2^21
    y, dig = fixed(fx, p, a, e)
    for i in range(a.shape[1]):
        v = sum(Fraction(int(dig[k, i])) * Fraction(2) ** (24 * (k + e)) for k in range(d))
        x = exact(a, i)
        assert abs(v) <= abs(x) and abs(x - v) < Fraction(2) ** (24 * e)   # truncation
        col = dig[:, i]
        assert np.all(np.abs(col) < 2 ** 24)
        assert np.all(col >= 0) or np.all(col <= 0)
        assert rel(exact(y, i), v) <= 2.0 ** (-53 * p + 2)


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("mode", [0, 1])
def test_dot_and_norm_by_diagonals(fx, p, mode):
    rng = np.random.default_rng(5 + mode)
    d = fx.fx_digits(p, 0)
    n = 300
    u, a = draw(rng, p, n, lo=-8, hi=1), draw(rng, p, n, lo=-8, hi=1)
    e = -(d - 1) + 1                                    # |entries| <= 2, norms <= 2^5
    out = np.zeros((p, 1))
    fx.fx_dot(p, mode, n, np.ascontiguousarray(u).ctypes.data_as(fx.dp),
              np.ascontiguousarray(a).ctypes.data_as(fx.dp), e, e, out.ctypes.data_as(fx.dp))
    # exact sum over the fixed-point values of the entries
    _, du = fixed(fx, p, u, e)
    _, da = fixed(fx, p, a, e)
    val = lambda dig, i: sum(int(dig[k, i]) << (24 * k) for k in range(d))
    want = sum((val(du, i) if mode == 0 else val(da, i)) * val(da, i) for i in range(n))
    want = Fraction(want) * Fraction(2) ** (48 * e)
    absmag = sum(abs(val(du if mode == 0 else da, i) * val(da, i)) for i in range(n)) * Fraction(2) ** (48 * e)
    dropped = n * d * Fraction(2) ** (48 + 24 * (d - 4) + 48 * e)   # diagonals below D-3
    err = abs(exact(out, 0) - want)
    assert err <= dropped + Fraction(2) ** (-53 * p + 2) * absmag


@pytest.mark.parametrize("p", PS)
def test_reflector_update(fx, p):
    """a -= w u with w as two integer and D-2 fractional digits of
    w 2^(24(eu-ea)); u on a finer scale than a (a rescaled Householder
    vector) and w large, as after the rescaling of a small reflector."""
    rng = np.random.default_rng(6)
    d = fx.fx_digits(p, 0)
    n = 100
    ea, eu = -(d - 1), -(d - 1) - 2                     # u two digits finer
    a = draw(rng, p, n, lo=-4, hi=0)
    u = draw(rng, p, n, lo=-6, hi=0) * 2.0 ** -48       # |u| < 2^-48
    w = draw(rng, p, 1, lo=40, hi=44)                   # w u stays below 2^-4
    a0 = a.copy()
    ok = fx.fx_axpy(p, n, a.ctypes.data_as(fx.dp), np.ascontiguousarray(u).ctypes.data_as(fx.dp),
                    np.ascontiguousarray(w).ctypes.data_as(fx.dp), ea, eu)
    assert ok == 1
    W = exact(w, 0)
    for i in range(n):
        want = exact(a0, i) - W * exact(u, i)
        # digit truncation of a, u (2^(24 ea), 2^(24 eu) * |w|), of w's fraction, final rounding
        bound = 4 * Fraction(2) ** (24 * ea) + abs(W) * Fraction(2) ** (24 * eu) \
            + Fraction(2) ** (-53 * p + 2) * abs(want)
        assert abs(exact(a, i) - want) <= bound, i


def test_update_refuses_a_multiplier_that_does_not_fit(fx):
    p = 4
    d = fx.fx_digits(p, 0)
    a = np.zeros((p, 4))
    u = np.zeros((p, 4))
    w = np.zeros((p, 1))
    w[0, 0] = 2.0 ** 60                                 # needs more than two integer digits
    assert fx.fx_axpy(p, 4, a.ctypes.data_as(fx.dp), u.ctypes.data_as(fx.dp),
                      w.ctypes.data_as(fx.dp), -(d - 1), -(d - 1)) == 0


@pytest.mark.parametrize("p,variant", [(p, v) for p in PS for v in ("digits", "md")] + [(2, "dd")])
def test_householder_scalars(fx, p, variant):
    """Golub and Van Loan's house() with the unscaled vector: mu = sqrt(x0^2 +
    sigma), v0 = x0 - mu, bp = -1/(mu v0) = 2/||u||^2, beta = bp v0^2, 1/v0;
    and the two degenerate kinds for sigma = 0.  Three forms: Newton on
    digits (within a few units of 2^(-53P)), P-limb FP64 arithmetic
    (xf_house_md, within 2^(10-53P): a handful of md operations, each with a
    relative error of a few units of 2^(-53P)), and the short-chain double
    double form of the panels (xf_house_dd: Newton-corrected reciprocals and
    root, products, the same bound)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 53 * p + 200
    rng = np.random.default_rng(11)
    n = 60
    sig = np.abs(draw(rng, p, n, lo=-10, hi=10)) * 1.0
    sig = sig * np.sign(sig[0])
    x0 = draw(rng, p, n, lo=-12, hi=12)
    sig[:, :4] = 0.0                                     # degenerate kinds
    x0[:, 1] = -x0[:, 1] * np.sign(x0[0, 1])             # negative x0 with sigma = 0
    x0[:, 2] = 0.0
    x0[:, 5] = 0.0                                       # x0 = 0 with sigma > 0
    outs = [np.zeros((p, n)) for _ in range(5)]
    kind = np.zeros(n, dtype=np.int32)
    args = [sig.ctypes.data_as(fx.dp), x0.ctypes.data_as(fx.dp),
            *[o.ctypes.data_as(fx.dp) for o in outs], kind.ctypes.data_as(C.POINTER(C.c_int))]
    if variant == "dd":
        fx.fx_house_dd(n, *args)
    else:
        (fx.fx_house if variant == "digits" else fx.fx_house_md)(p, n, *args)
    v0, bp, rcc, inv, beta = outs
    mp = lambda x, i: mpmath.fsum([mpmath.mpf(float(v)) for v in x[:, i]])
    tol = mpmath.mpf(2) ** (-53 * p + (6 if variant == "digits" else 10))
    for i in range(n):
        s, x = mp(sig, i), mp(x0, i)
        if s == 0:
            assert kind[i] == (1 if x >= 0 else 2)
            assert mp(v0, i) == 1 and mp(inv, i) == 1
            assert mp(bp, i) == (0 if x >= 0 else 2) and mp(beta, i) == mp(bp, i)
            assert abs(mp(rcc, i) - abs(x)) <= tol * abs(x)
            continue
        assert kind[i] == 0
        mu = mpmath.sqrt(x * x + s)
        want_v0 = x - mu if x <= 0 else -s / (x + mu)
        checks = [(rcc, mu), (v0, want_v0), (bp, -1 / (mu * want_v0)), (inv, 1 / want_v0),
                  (beta, -want_v0 / mu)]
        for got, want in checks:
            assert abs(mp(got, i) - want) <= tol * abs(want), (i, got is v0)


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("m,n", [(12, 12), (40, 33), (9, 5)])
def test_panel_replay_matches_oracle_qr(fx, p, m, n):
    """The integer-digit panel's steps, replayed sequentially on the host for
    one panel holding every column, give the oracle's unblocked Householder
    QR: R, the Householder vectors below the diagonal and the betas."""
    import oracle
    import synth
    A, _ = synth.lstsq_problem(p, m, n, seed=21, tag="fxpanel")
    A = np.ascontiguousarray(A)
    R_ref, _, beta_ref = oracle.qr(A, want_q=False)
    W = A.copy()
    beta = np.zeros((p, n))
    rc = fx.fx_panel_replay(p, m, n, W.ctypes.data_as(fx.dp), beta.ctypes.data_as(fx.dp))
    assert rc == 0
    tol = {2: 1e-28, 4: 1e-60, 8: 1e-118}[p]
    upper = np.triu(np.ones((m, n), dtype=bool)).T      # (n, m) mask of R's entries
    assert oracle.rel_err(np.where(upper, W, 0.0), R_ref) < tol
    assert oracle.rel_err(beta, beta_ref) < tol
