"""Operation counts: the flop convention of every TFLOPS figure.

Table 1 of arXiv 2110.08375 (Section 1.1) gives the double-precision operation
count of one md add, mul and div; the paper converts per-kernel tallies of md
operations to flops with these multipliers.  Here the md operations tallied
are those of the UNBLOCKED Householder algorithm (the method's plain
definition, column by column), so the blocked algorithm's extra work (the WY
matrices, inverted diagonal tiles) earns no credit.  A square root counts as
one division; a subtraction as one addition.

Also here: the FP64 instruction and flop counts of one device md operation as
the kernels implement them (csrc/md.cuh, "bins by order"), used for the FP64
roofline.  FLOPs count an FMA as 2.
"""
from __future__ import annotations

TABLE1_SIGMA = {2: {"add": 20, "mul": 23, "div": 70},
                4: {"add": 89, "mul": 336, "div": 893},
                8: {"add": 269, "mul": 1742, "div": 5126}}


def table1_flops(p: int, counts: dict) -> int:
    t = TABLE1_SIGMA[p]
    return (counts.get("add", 0) * t["add"] + counts.get("mul", 0) * t["mul"]
            + (counts.get("div", 0) + counts.get("sqrt", 0)) * t["div"])


def qr_counts(m: int, n: int, want_q: bool = False, extra_cols: int = 0) -> dict:
    """md operations of unblocked Householder QR of an m x n matrix, applied
    also to ``extra_cols`` right-hand sides, Q accumulated when ``want_q``.

    Column j (L = m - j rows): sigma = sum of squares, L-1 mul + L-1 add; when
    L > 1 the reflector (mu, v0, beta, v) costs 2 mul + 3 add + 1 sqrt + L div
    (the extra division of the x0 > 0 branch is not counted); applying it to
    one column costs 2L+1 mul + 2L add.  The last column of a square matrix
    (L = 1) has no reflector.
    """
    add = mul = dv = sq = 0
    for j in range(n):
        L = m - j
        mul += L - 1
        add += L - 1
        if L == 1:
            continue
        mul += 2
        add += 3
        sq += 1
        dv += L
        cols = (n - j - 1) + extra_cols + ((m - j) if want_q else 0)
        mul += cols * (2 * L + 1)
        add += cols * (2 * L)
    return {"add": add, "mul": mul, "div": dv, "sqrt": sq}


def backsub_counts(n: int) -> dict:
    """Row-by-row back substitution: n(n-1)/2 mul and add, n div."""
    return {"add": n * (n - 1) // 2, "mul": n * (n - 1) // 2, "div": n, "sqrt": 0}


def lstsq_counts(m: int, n: int) -> dict:
    """QR of [A | b] (no Q) followed by back substitution."""
    q = qr_counts(m, n, want_q=False, extra_cols=1)
    b = backsub_counts(n)
    return {k: q[k] + b[k] for k in q}


def lstsq_table1_flops(p: int, m: int, n: int) -> int:
    return table1_flops(p, lstsq_counts(m, n))


def toeplitz_counts(m: int, n: int, d: int) -> dict:
    """md operations of the block-Toeplitz solve by block forward
    substitution: the QR of J_0 (no Q), then for every block k = 0..d the
    residual b_k - sum_{i=1}^{k} J_i x_{k-i} (k m n multiply-adds), Q^T r
    (the n reflectors applied to one vector: 2L+1 mul and 2L add for a
    reflector of length L) and the back substitution."""
    q = qr_counts(m, n, want_q=False)
    add = mul = 0
    for j in range(n):
        L = m - j
        if L > 1:
            mul += 2 * L + 1
            add += 2 * L
    bs = backsub_counts(n)
    res = (d * (d + 1) // 2) * m * n
    blocks = d + 1
    return {"add": q["add"] + blocks * (add + bs["add"]) + res,
            "mul": q["mul"] + blocks * (mul + bs["mul"]) + res,
            "div": q["div"] + blocks * bs["div"], "sqrt": q["sqrt"]}


def complex_counts(real: dict) -> dict:
    """md operations of the complex algorithm from those of the real one:
    a complex multiplication is 4 md multiplications and 2 md additions, a
    complex addition 2 md additions, so each real multiply-add of the
    unblocked algorithm becomes 4 md multiplications and 4 md additions (the
    paper: complex data take about four times as many operations); the
    divisions and square roots of the reflectors are counted as in the real
    algorithm (lower order terms)."""
    return {"add": 4 * real["add"], "mul": 4 * real["mul"], "div": real["div"], "sqrt": real["sqrt"]}


def zqr_table1_flops(p: int, m: int, n: int, want_q: bool = True) -> int:
    return table1_flops(p, complex_counts(qr_counts(m, n, want_q=want_q)))


def zlstsq_table1_flops(p: int, m: int, n: int) -> int:
    return table1_flops(p, complex_counts(lstsq_counts(m, n)))


# ---------------------------------------------------------------------------
# FP64 cost of one device md operation (csrc/md.cuh)
# ---------------------------------------------------------------------------
TWO_SUM_INT = (1, 1)   # (instructions, flops): the FP64 addition; its exact error on the integer pipe
TWO_SUM_FAST = (3, 3)  # Fast2Sum, the operand order taken on the integer pipe
TWO_PROD = (2, 3)     # DMUL + DFMA
DFMA = (1, 2)
DADD = (1, 1)


def _add(a, b, k=1):
    return (a[0] + k * b[0], a[1] + k * b[1])


def two_sum_cost(p: int, d: int):
    """The two_sum form bin d of a p-limb operation uses (csrc/md.cuh,
    two_sum_pd): the integer error for p <= 4 and for the first five bins of
    od; renormalisation counts as bin p."""
    return TWO_SUM_INT if (p <= 4 or d < 5) else TWO_SUM_FAST


def renorm_cost(p: int):
    n = (p - 1) + (p - 2 if p > 2 else 0)
    ts = two_sum_cost(p, p)
    return (n * ts[0], n * ts[1])


def fma_cost(p: int, with_c: bool = True):
    """(FP64 instructions, FP64 flops) of md c + a*b (with_c) or a*b."""
    cost = (0, 0)
    ne = 0
    for d in range(p):
        nlo = d
        if d < p - 1:
            nterms = (1 if with_c else 0) + (d + 1) + nlo + ne
            cost = _add(cost, TWO_PROD, d + 1)
            cost = _add(cost, two_sum_cost(p, d), nterms - 1)
            ne = nterms - 1
        else:
            cost = _add(cost, DFMA, d + 1)
            cost = _add(cost, DADD, nlo + ne)
    return _add(cost, renorm_cost(p))


def gemm_fma_cost(p: int, renorm_every: int = 16):
    """FP64 instructions per md FMA of the product loops (csrc/kernels.cuh:
    md_fma_bins, one renormalisation per `renorm_every` steps)."""
    full = fma_cost(p)[0]
    rn = renorm_cost(p)[0]
    return full - rn + rn / renorm_every


def add_cost(p: int):
    cost = (0, 0)
    ne = 0
    for d in range(p):
        if d < p - 1:
            cost = _add(cost, two_sum_cost(p, d), 1 + ne)
            ne += 1
        else:
            cost = _add(cost, DADD, 1 + ne)
    return _add(cost, renorm_cost(p))


def gemm_md_fmas(M: int, N: int, K: int) -> int:
    """md FMAs of one M x N x K product (one per output per k)."""
    return M * N * K


def trailing_md_fmas(m: int, n: int, t: int, extra_cols: int = 0) -> int:
    """md FMAs of the trailing updates X = W^T C (w x nc x r) and
    C += Y X (r x nc x w) over all tiles of a blocked QR."""
    total = 0
    for j0 in range(0, n, t):
        w = min(t, n - j0)
        r = m - j0
        nc = n + extra_cols - (j0 + w)
        if nc > 0:
            total += 2 * w * nc * r
    return total


def wy_md_fmas(m: int, n: int, t: int, extra_cols: int = 0) -> int:
    """md FMAs of the WY form's two products over all tiles that have a
    trailing update: G = Y^T Y (upper triangle, w (w+1)/2 outputs of r
    terms) and W = -Y T (T upper triangular: r x w outputs, j + 1 terms for
    column j)."""
    total = 0
    for j0 in range(0, n, t):
        w = min(t, n - j0)
        r = m - j0
        if n + extra_cols - (j0 + w) > 0:
            total += 2 * (w * (w + 1) // 2) * r
    return total
