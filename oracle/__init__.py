"""CPU oracle for multiple-double least squares (arXiv 2110.08375).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  The product library never
imports, links or executes anything here, and the two share no code.

The arithmetic lives in ``mdref.c`` (C, built with gcc, no fast-math and no
FP contraction); this module only marshals numpy arrays to it.  Arrays use the
limb-planar layout of the paper's Section 2: an md matrix with ``rows x cols``
entries is a float64 array of shape ``(p, cols, rows)``, a vector ``(p, n)``.

Every function here is pinned by the ``-m "not gpu"`` tests: md arithmetic
against exact rational arithmetic (``fractions.Fraction``) and high-precision
decimals, QR and least squares against exact rational solutions of small
systems, invariants (orthogonality, A = QR, normal equations) and special
cases, and the operation counters against closed forms.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdref.c")
LIB = os.path.join(HERE, "libmdref.so")

_lib = None
_dp = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compiles mdref.c into libmdref.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "mdref.h"))):
        return LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        i64 = C.c_int64
        L.mdref_two_sum.argtypes = [C.c_double, C.c_double, _dp, _dp]
        L.mdref_two_prod.argtypes = [C.c_double, C.c_double, _dp, _dp]
        for name in ("mdref_add", "mdref_sub", "mdref_mul", "mdref_div"):
            getattr(L, name).argtypes = [C.c_int, _dp, _dp, _dp]
        L.mdref_sqrt.argtypes = [C.c_int, _dp, _dp]
        L.mdref_normalize.argtypes = [C.c_int, _dp, _dp]
        L.mdref_diff.argtypes = [C.c_int, _dp, _dp]
        L.mdref_diff.restype = C.c_double
        L.mdref_diff_array.argtypes = [C.c_int, i64, _dp, i64, _dp, i64, _dp]
        L.mdref_get_counts.argtypes = [C.POINTER(C.c_uint64)]
        L.mdref_set_threads.argtypes = [C.c_int]
        L.mdref_qr.argtypes = [C.c_int, i64, i64, _dp, i64, i64, _dp, i64, i64, _dp]
        L.mdref_backsub.argtypes = [C.c_int, i64, _dp, i64, i64, _dp, _dp]
        L.mdref_lstsq.argtypes = [C.c_int, i64, i64, _dp, i64, i64, _dp, _dp]
        L.mdref_gemv.argtypes = [C.c_int, C.c_int, i64, i64, _dp, i64, i64, _dp, _dp]
        L.mdref_gemm.argtypes = [C.c_int, i64, i64, i64, _dp, i64, i64, _dp, i64, i64, _dp,
                                 i64, i64]
        L.mdref_zqr.argtypes = [C.c_int, i64, i64, _dp, _dp, i64, i64, _dp, _dp, i64, i64, _dp]
        L.mdref_zbacksub.argtypes = [C.c_int, i64, _dp, _dp, i64, i64, _dp, _dp, _dp, _dp]
        L.mdref_zlstsq.argtypes = [C.c_int, i64, i64, _dp, _dp, i64, i64, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _md(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    lib().mdref_set_threads(int(n))


def threads() -> int:
    return lib().mdref_get_threads()


def two_sum(a: float, b: float):
    s, e = C.c_double(), C.c_double()
    lib().mdref_two_sum(a, b, C.byref(s), C.byref(e))
    return s.value, e.value


def two_prod(a: float, b: float):
    s, e = C.c_double(), C.c_double()
    lib().mdref_two_prod(a, b, C.byref(s), C.byref(e))
    return s.value, e.value


def _binop(name, a, b):
    a, b = _md(a), _md(b)
    c = np.zeros_like(a)
    getattr(lib(), name)(a.size, _ptr(a), _ptr(b), _ptr(c))
    return c


def add(a, b):
    return _binop("mdref_add", a, b)


def sub(a, b):
    return _binop("mdref_sub", a, b)


def mul(a, b):
    return _binop("mdref_mul", a, b)


def div(a, b):
    return _binop("mdref_div", a, b)


def sqrt(a):
    a = _md(a)
    c = np.zeros_like(a)
    lib().mdref_sqrt(a.size, _ptr(a), _ptr(c))
    return c


def normalize(a):
    a = _md(a)
    c = np.zeros_like(a)
    lib().mdref_normalize(a.size, _ptr(a), _ptr(c))
    return c


def diff(a, b) -> np.ndarray:
    """RN(a - b) elementwise for md arrays of shape (p, ...) (exact before rounding)."""
    a, b = _md(a), _md(b)
    assert a.shape == b.shape
    p = a.shape[0]
    cnt = a[0].size
    out = np.zeros(cnt, dtype=np.float64)
    lib().mdref_diff_array(p, cnt, _ptr(a), cnt, _ptr(b), cnt, _ptr(out))
    return out.reshape(a.shape[1:])


def rel_err(x, ref) -> float:
    """||x - ref||_2 / ||ref||_2 with the difference formed exactly."""
    d = diff(x, ref)
    nr = float(np.linalg.norm(_md(ref)[0].ravel()))
    nd = float(np.linalg.norm(d.ravel()))
    return nd / nr if nr else nd


def reset_counts() -> None:
    lib().mdref_reset_counts()


def counts() -> dict:
    out = (C.c_uint64 * 7)()
    lib().mdref_get_counts(out)
    keys = ("add", "mul", "div", "sqrt", "pos_branch", "ident", "flip")
    return dict(zip(keys, [int(v) for v in out]))


def qr(A, want_q: bool = True):
    """Householder QR.  A: (p, n, m) limb-planar.  Returns (R, Q or None, beta)."""
    A = _md(A).copy()
    p, n, m = A.shape
    Q = np.zeros((p, m, m)) if want_q else None
    beta = np.zeros((p, n))
    rc = lib().mdref_qr(p, m, n, _ptr(A), m, n * m, _ptr(Q) if want_q else None,
                        m, m * m, _ptr(beta))
    if rc:
        raise ValueError(f"mdref_qr failed: {rc}")
    return A, Q, beta


def backsub(R, y):
    """Solves R x = y for R (p, n, ld) upper triangular (leading n x n used)."""
    R, y = _md(R), _md(y)
    p, n, ld = R.shape
    x = np.zeros((p, n))
    rc = lib().mdref_backsub(p, n, _ptr(R), ld, n * ld, _ptr(y), _ptr(x))
    if rc:
        raise ZeroDivisionError("zero diagonal entry in R")
    return x


def lstsq(A, b):
    A, b = _md(A), _md(b)
    p, n, m = A.shape
    x = np.zeros((p, n))
    rc = lib().mdref_lstsq(p, m, n, _ptr(A), m, n * m, _ptr(b), _ptr(x))
    if rc == -2:
        raise ZeroDivisionError("zero diagonal entry in R")
    if rc:
        raise ValueError(f"mdref_lstsq failed: {rc}")
    return x


def zqr(Ar, Ai, want_q: bool = True):
    """Complex Householder QR (Hermitian reflectors, diag(R) = phase(x0) ||x||).
    Ar, Ai: (p, n, m) limb-planar real and imaginary parts.  Returns
    (Rr, Ri, Qr, Qi, beta) with Q None when want_q is False."""
    Ar, Ai = _md(Ar).copy(), _md(Ai).copy()
    p, n, m = Ar.shape
    Qr = np.zeros((p, m, m)) if want_q else None
    Qi = np.zeros((p, m, m)) if want_q else None
    beta = np.zeros((p, n))
    rc = lib().mdref_zqr(p, m, n, _ptr(Ar), _ptr(Ai), m, n * m, _ptr(Qr) if want_q else None,
                         _ptr(Qi) if want_q else None, m, m * m, _ptr(beta))
    if rc:
        raise ValueError(f"mdref_zqr failed: {rc}")
    return Ar, Ai, Qr, Qi, beta


def zbacksub(Rr, Ri, yr, yi):
    """Solves R x = y for complex upper triangular R (re/im planes (p, n, ld))."""
    Rr, Ri, yr, yi = _md(Rr), _md(Ri), _md(yr), _md(yi)
    p, n, ld = Rr.shape
    xr, xi = np.zeros((p, n)), np.zeros((p, n))
    rc = lib().mdref_zbacksub(p, n, _ptr(Rr), _ptr(Ri), ld, n * ld, _ptr(yr), _ptr(yi), _ptr(xr), _ptr(xi))
    if rc:
        raise ZeroDivisionError("zero diagonal entry in R")
    return xr, xi


def zlstsq(Ar, Ai, br, bi):
    """Complex least squares: min ||b - A x|| (unblocked complex Householder QR of [A | b])."""
    Ar, Ai, br, bi = _md(Ar), _md(Ai), _md(br), _md(bi)
    p, n, m = Ar.shape
    xr, xi = np.zeros((p, n)), np.zeros((p, n))
    rc = lib().mdref_zlstsq(p, m, n, _ptr(Ar), _ptr(Ai), m, n * m, _ptr(br), _ptr(bi), _ptr(xr), _ptr(xi))
    if rc == -2:
        raise ZeroDivisionError("zero diagonal entry in R")
    if rc:
        raise ValueError(f"mdref_zlstsq failed: {rc}")
    return xr, xi


def toeplitz_lstsq(J, b):
    """Block forward substitution of the lower triangular block-Toeplitz
    system J(t) x(t) = b(t) mod t^{d+1}: x_k = lstsq(J_0, b_k - sum_{i=1}^{k}
    J_i x_{k-i}) for k = 0..d, every step in md arithmetic (the residual by
    gemv and elementwise subtraction, each block by the unblocked
    Householder least squares).  J: (p, d+1, n, m), b: (p, d+1, m); returns
    x (p, d+1, n)."""
    J, b = _md(J), _md(b)
    p, d1, n, m = J.shape
    x = np.zeros((p, d1, n))
    for k in range(d1):
        r = b[:, k].copy()
        for i in range(1, k + 1):
            r = _vec_sub(r, gemv(J[:, i], x[:, k - i]))
        x[:, k] = lstsq(J[:, 0], r)
    return x


def zrel_err(xr, xi, rr, ri) -> float:
    """||x - ref|| / ||ref|| for complex md arrays, differences formed exactly."""
    dr, di = diff(xr, rr), diff(xi, ri)
    nr = float(np.sqrt(np.sum(_md(rr)[0] ** 2) + np.sum(_md(ri)[0] ** 2)))
    nd = float(np.sqrt(np.sum(dr ** 2) + np.sum(di ** 2)))
    return nd / nr if nr else nd


def gemv(A, x, trans: bool = False):
    A, x = _md(A), _md(x)
    p, n, m = A.shape
    y = np.zeros((p, n if trans else m))
    lib().mdref_gemv(p, int(trans), m, n, _ptr(A), m, n * m, _ptr(x), _ptr(y))
    return y


def gemm(A, B):
    """C = A B for limb-planar A (p, k, m), B (p, n, k); returns (p, n, m)."""
    A, B = _md(A), _md(B)
    p, k, m = A.shape
    _, n, k2 = B.shape
    assert k == k2
    Cm = np.zeros((p, n, m))
    lib().mdref_gemm(p, m, n, k, _ptr(A), m, k * m, _ptr(B), k, n * k, _ptr(Cm), m, n * m)
    return Cm


def residual(A, x, b):
    """r = b - A x, every operation in md arithmetic."""
    return _vec_sub(b, gemv(A, x))


def _vec_sub(a, b):
    a, b = _md(a), _md(b)
    p = a.shape[0]
    out = np.zeros_like(a)
    for i in range(a.shape[1]):
        out[:, i] = sub(a[:, i], b[:, i])
    return out


# flop convention: double operations per md operation, from the paper's
# Table 1 (columns +, -, *, / and their sum)
TABLE1 = {
    2: {"add": (8, 12, 0, 0, 20), "mul": (5, 9, 9, 0, 23), "div": (33, 18, 16, 3, 70)},
    4: {"add": (35, 54, 0, 0, 89), "mul": (99, 164, 73, 0, 336), "div": (266, 510, 112, 5, 893)},
    8: {"add": (95, 174, 0, 0, 269), "mul": (529, 954, 259, 0, 1742),
        "div": (1599, 3070, 448, 9, 5126)},
}


def table1_flops(p: int, n_add: int, n_mul: int, n_div: int, n_sqrt: int = 0) -> int:
    """Double-precision operations for the given md operation counts (Table 1
    multipliers; a square root is counted as one division)."""
    t = TABLE1[p]
    return n_add * t["add"][4] + n_mul * t["mul"][4] + (n_div + n_sqrt) * t["div"][4]


def qr_counts_closed_form(m: int, n: int, want_q: bool, npos: int = 0, degenerate=(),
                          ident=(), extra_cols: int = 0) -> dict:
    """md operation counts of :func:`qr` / the QR part of :func:`lstsq`
    (unblocked, as coded in mdref.c).

    Per column j (L = m - j): sigma costs L-1 mul + L-1 add.  When sigma != 0
    the reflector costs mu (1 mul, 1 add, 1 sqrt), v0 (1 add, plus 1 div on
    the x0 > 0 branch, counted by ``npos``), beta (1 mul, 1 add, 1 div) and
    v (L-1 div).  ``degenerate`` lists the columns with sigma == 0 and
    ``ident`` those of them whose reflector is the identity (x0 >= 0); an
    identity reflector is applied to nothing.  Applying a reflector to one
    column of length L costs 2L+1 mul and 2L add; it is applied to the n-j-1
    trailing columns, to ``extra_cols`` right-hand sides, and (with Q) to the
    m-j columns j..m-1 of Q in the backward accumulation.
    """
    add = mul = dv = sq = 0
    degenerate, ident = set(degenerate), set(ident)
    for j in range(n):
        L = m - j
        mul += L - 1
        add += L - 1
        if j not in degenerate:
            mul += 2
            add += 3
            sq += 1
            dv += 1 + (L - 1)
        if j in ident:
            continue
        ncols = (n - j - 1) + extra_cols
        if want_q:
            ncols += m - j
        mul += ncols * (2 * L + 1)
        add += ncols * (2 * L)
    dv += npos
    return {"add": add, "mul": mul, "div": dv, "sqrt": sq}


def backsub_counts_closed_form(n: int) -> dict:
    return {"add": n * (n - 1) // 2, "mul": n * (n - 1) // 2, "div": n, "sqrt": 0}
