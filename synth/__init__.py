"""Seeded synthetic inputs for the multiple-double least-squares path.

This module is shared by the CPU oracle side (tests) and the CUDA side
(tests, bench).  It draws random numbers and lays them out; it performs no
multiple-double arithmetic at all (no sums of limbs, no renormalisation, no
products of matrices).

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), one stream per (seed, label).  A draw
``z`` becomes ``u = (z >> 11) * 2**-53`` in [0, 1), and ``2u - 1`` in [-1, 1).

Multiple-double values (p limbs, most significant first) are drawn as
``x0 ~ U[-1,1)`` and ``x_i = x_{i-1} * 2**-54 * U[-1,1)``.  Each lower limb is
therefore strictly below half an ulp of the limb above it, so the limbs are
already normalised and no arithmetic is needed to make them so.

Layout: limb-planar ("staggered" storage of the paper's Section 2): an md
matrix with ``rows x cols`` entries is a float64 array of shape
``(p, cols, rows)`` -- p planes, each column-major.  A vector of length n is
``(p, n)``.
"""
from __future__ import annotations

import math
import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

PRECISIONS = {"dd": 2, "qd": 4, "od": 8}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _fnv1a64(label: str) -> int:
    h = 0xCBF29CE484222325
    for ch in label.encode():
        h ^= ch
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def stream_seed(seed: int, label: str) -> int:
    """64-bit start state of the stream named ``label`` under ``seed``."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN_GAMMA
        s = s ^ np.uint64(_fnv1a64(label))
        return int(_mix(np.array([s], dtype=np.uint64))[0])


def splitmix64(state: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream at ``state``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(state) + idx * GOLDEN_GAMMA
        return _mix(z)


def unit(seed: int, label: str, count: int, offset: int = 0) -> np.ndarray:
    """``count`` draws of U[0, 1) (multiples of 2**-53)."""
    z = splitmix64(stream_seed(seed, label), count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sym(seed: int, label: str, count: int, offset: int = 0) -> np.ndarray:
    """``count`` draws of U[-1, 1)."""
    return 2.0 * unit(seed, label, count, offset) - 1.0


def md_limbs_from_top(top: np.ndarray, p: int, seed: int, label: str) -> np.ndarray:
    """Attaches p-1 lower limbs to the top limbs ``top`` (any shape).

    Returns shape ``(p,) + top.shape``; limb i is limb i-1 times 2**-54 times
    a fresh U[-1,1) draw, which keeps it under half an ulp of limb i-1.
    """
    out = np.empty((p,) + top.shape, dtype=np.float64)
    out[0] = top
    n = top.size
    for i in range(1, p):
        r = sym(seed, f"{label}/limb{i}", n).reshape(top.shape)
        out[i] = out[i - 1] * (2.0 ** -54) * r
    return out


def md_uniform(p: int, shape: tuple, seed: int, label: str) -> np.ndarray:
    """md values with top limb ~ U[-1,1); shape ``(p,) + shape``."""
    n = int(np.prod(shape)) if len(shape) else 1
    top = sym(seed, f"{label}/limb0", n).reshape(shape)
    return md_limbs_from_top(top, p, seed, label)


def md_matrix(p: int, rows: int, cols: int, seed: int, label: str) -> np.ndarray:
    """rows x cols md matrix, entries ~ U[-1,1) (limb-planar, (p, cols, rows))."""
    return np.ascontiguousarray(md_uniform(p, (cols, rows), seed, label))


def md_vector(p: int, n: int, seed: int, label: str) -> np.ndarray:
    return np.ascontiguousarray(md_uniform(p, (n,), seed, label))


# ----------------------------------------------------------------------------
# Workloads.  Shapes and distributions follow the five benchmark configurations
# of this project (dense least squares, precision modes, back substitution,
# batched).  Every function is deterministic in ``seed``.
# ----------------------------------------------------------------------------

def lstsq_problem(p: int, m: int, n: int, seed: int = 0, tag: str = "ls"):
    """Dense A (m x n) and b (m), entries ~ U[-1,1) in every limb recipe."""
    A = md_matrix(p, m, n, seed, f"{tag}/A/{m}x{n}/p{p}")
    b = md_vector(p, m, seed, f"{tag}/b/{m}/p{p}")
    return A, b


def upper_triangular(p: int, n: int, seed: int = 0, tag: str = "bs", ld: int | None = None):
    """Upper triangular R (n x n) with diag ~ U[1,2], strict upper ~ U[-1,1)/n.

    Entries below the diagonal are zero.  Returns (R, y) with y ~ U[-1,1).
    ``ld`` pads each column (rows beyond n are zero).
    """
    ld = n if ld is None else ld
    top = np.zeros((n, ld), dtype=np.float64)          # [col][row]
    for j in range(n):
        if j:
            top[j, :j] = sym(seed, f"{tag}/R/{n}/off", j, offset=j * (j - 1) // 2) / n
        top[j, j] = 1.0 + unit(seed, f"{tag}/R/{n}/diag", 1, offset=j)[0]
    R = md_limbs_from_top(top, p, seed, f"{tag}/R/{n}/p{p}")
    R[:, :, n:] = 0.0
    for j in range(n):                                   # keep the lower part exactly zero
        R[:, j, j + 1:] = 0.0
    y = md_vector(p, n, seed, f"{tag}/y/{n}/p{p}")
    return np.ascontiguousarray(R), y


def upper_triangular_fast(p: int, n: int, seed: int = 0, tag: str = "bs"):
    """Same distribution as :func:`upper_triangular` for large n, built column
    block by column block without Python loops over rows (used for n in the
    ten-thousands).  Strict-upper entries come from one stream indexed by the
    packed position j*(j-1)/2 + i, so both builders give identical matrices."""
    R = np.zeros((p, n, n), dtype=np.float64)
    off_state = stream_seed(seed, f"{tag}/R/{n}/off")
    diag = 1.0 + unit(seed, f"{tag}/R/{n}/diag", n)
    step = 512
    for j0 in range(0, n, step):
        j1 = min(n, j0 + step)
        cols = np.arange(j0, j1)
        start = j0 * (j0 - 1) // 2 if j0 else 0
        count = j1 * (j1 - 1) // 2 - start
        z = splitmix64(off_state, count, start)
        vals = (2.0 * ((z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)) - 1.0) / n
        blk = np.zeros((j1 - j0, n), dtype=np.float64)
        pos = 0
        for jj, j in enumerate(cols):
            blk[jj, :j] = vals[pos:pos + j]
            pos += j
            blk[jj, j] = diag[j]
        R[0, j0:j1] = blk
    for i in range(1, p):
        for j0 in range(0, n, step):
            j1 = min(n, j0 + step)
            cnt = (j1 - j0) * n
            r = sym(seed, f"{tag}/R/{n}/p{p}/limb{i}", cnt, offset=j0 * n).reshape(j1 - j0, n)
            R[i, j0:j1] = R[i - 1, j0:j1] * (2.0 ** -54) * r
    y = md_vector(p, n, seed, f"{tag}/y/{n}/p{p}")
    return R, y


def batched_shapes(count: int = 512, seed: int = 0, nmin: int = 32, nmax: int = 512):
    """Shapes and precisions of the batched workload.

    n = floor(exp(U[ln nmin, ln nmax])), m = n + U{0..n}; the first half of the
    problems are double double (p=2), the second half quad double (p=4), and
    the order is shuffled by a seeded permutation.
    """
    u = unit(seed, "batch/n", count)
    n = np.floor(np.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))).astype(np.int64)
    n = np.clip(n, nmin, nmax)
    um = unit(seed, "batch/m", count)
    m = n + np.floor(um * (n + 1)).astype(np.int64)
    p = np.where(np.arange(count) < count // 2, 2, 4)
    key = unit(seed, "batch/perm", count)
    perm = np.argsort(key, kind="stable")
    return [(int(m[i]), int(n[i]), int(p[i])) for i in perm]


def batched_problem(idx: int, m: int, n: int, p: int, seed: int = 0):
    return lstsq_problem(p, m, n, seed, tag=f"batch{idx}")


# ----------------------------------------------------------------------------
# Precision-mode workload: A = U diag(sigma) V^T with exactly orthogonal U, V
# and singular values log-spaced over a chosen condition number.
#
# With Sylvester's Hadamard matrix H_N (entries (-1)^popcount(i & j)):
#   U = D_u H_m[:, c] / sqrt(m)   (n columns of the randomised H_m: D_u random
#                                  signs, c a seeded random subset of columns),
#   V^T = H_n[pi, :] D_v / sqrt(n) (pi a seeded permutation, D_v random signs),
#   sigma_k = d_k / sqrt(2), d_k = D_k 2^-20, D_k = round(2^20 kappa^(k/(n-1))).
# U and V are exactly orthogonal.  For m = 4^a and n = 2 * 4^b the scale
# sqrt(2) / (sqrt(m) sqrt(n)) is a power of two, so every entry of
#   A = 2^-shift_a D_u H_m[:, c] diag(D) H_n[pi, :] D_v
# is an exact dyadic number (an integer below 2^51 times 2^-shift_a), and
# kappa = max sigma / min sigma.  Only integer transforms are used (Walsh-
# Hadamard butterflies on int64 and on Python integers); every value is exact
# and the md values handed out are those exact numbers split into doubles by
# bit slicing (no rounding).
# ----------------------------------------------------------------------------

def _fwht_int64(Z: np.ndarray) -> np.ndarray:
    """H_N Z for Sylvester's H_N (N = Z.shape[0], a power of two), exact in
    int64 while the magnitudes stay below 2^63."""
    Z = Z.copy()
    N = Z.shape[0]
    h = 1
    while h < N:
        Z = Z.reshape(N // (2 * h), 2, h, *Z.shape[1:])
        a = Z[:, 0].copy()
        b = Z[:, 1]
        Z[:, 0] = a + b
        Z[:, 1] = a - b
        Z = Z.reshape(N, *Z.shape[3:])
        h *= 2
    return Z


def fwht_py(v: list) -> list:
    """H_N v for a list of Python integers (exact)."""
    v = list(v)
    N = len(v)
    h = 1
    while h < N:
        for s in range(0, N, 2 * h):
            for i in range(s, s + h):
                a, b = v[i], v[i + h]
                v[i], v[i + h] = a + b, a - b
        h *= 2
    return v


def split_exact(num: int, shift: int, p: int) -> list:
    """num * 2^-shift (a Python integer numerator) as p doubles by bit
    slicing: limb 0 holds the leading 53 bits, limb 1 the next 53, and so on
    (each limb below one ulp of the one above; exact when the value has at
    most 53 p significant bits, otherwise the bits beyond are dropped)."""
    import math
    out = [0.0] * p
    if num == 0:
        return out
    sgn = -1 if num < 0 else 1
    a = -num if num < 0 else num
    top = a.bit_length()
    for i in range(p):
        lo = top - 53 * (i + 1)
        if lo > 0:
            chunk = (a >> lo) & ((1 << 53) - 1)
            out[i] = sgn * math.ldexp(float(chunk), lo - shift)
        else:
            chunk = a & ((1 << (53 + lo)) - 1) if 53 + lo > 0 else 0
            out[i] = sgn * math.ldexp(float(chunk), -shift)
            break
    return out


def modes_structure(m: int = 4096, n: int = 2048, kappa: float = 1e6, seed: int = 0,
                    tag: str = "modes") -> dict:
    """The random choices of the precision-mode matrix (see above): signs
    du (m), dv (n), the column subset c (n of range(m)), the permutation pi
    (n) and the integer singular-value numerators D (n), with the scale
    exponents (A = 2^-shift_a D_u H_m[:, c] diag(D) H_n[pi, :] D_v)."""
    lm, ln = int(math.log2(m)), int(math.log2(n))
    if 2 ** lm != m or 2 ** ln != n or lm % 2 != 0 or ln % 2 != 1 or n > m:
        raise ValueError("needs m = 4^a >= n = 2 * 4^b")
    lab = f"{tag}/{m}x{n}/k{kappa:g}/s{seed}"
    du = np.where(unit(seed, lab + "/du", m) < 0.5, -1, 1).astype(np.int64)
    dv = np.where(unit(seed, lab + "/dv", n) < 0.5, -1, 1).astype(np.int64)
    c = np.sort(np.argsort(unit(seed, lab + "/c", m), kind="stable")[:n]).astype(np.int64)
    pi = np.argsort(unit(seed, lab + "/pi", n), kind="stable").astype(np.int64)
    k = np.arange(n, dtype=np.float64)
    D = np.rint(np.power(float(kappa), k / (n - 1)) * 2.0 ** 20).astype(np.int64)
    # 1/sqrt(m) = 2^-(lm/2) and 1/(sqrt(2) sqrt(n)) = 2^-((ln+1)/2); d = D 2^-20
    shift_a = lm // 2 + (ln + 1) // 2 + 20
    return {"m": m, "n": n, "kappa": kappa, "du": du, "dv": dv, "c": c, "pi": pi, "D": D,
            "shift_a": shift_a, "shift_sigma": 20}


def hadamard_rows(rows: np.ndarray, N: int) -> np.ndarray:
    """Rows `rows` of Sylvester's H_N as int64 (+-1): (-1)^popcount(r & j)."""
    j = np.arange(N, dtype=np.int64)
    par = (np.bitwise_count(rows[:, None] & j[None, :]) & 1).astype(np.int64)
    return 1 - 2 * par


def modes_matrix_int(st: dict) -> np.ndarray:
    """Integer numerators Aint (m x n, row-major [i][j]) with A = Aint 2^-shift_a."""
    m, n = st["m"], st["n"]
    M = hadamard_rows(st["pi"], n) * st["D"][:, None] * st["dv"][None, :]   # diag(D) H_n[pi, :] D_v
    Z = np.zeros((m, n), dtype=np.int64)
    Z[st["c"]] = M
    Y = _fwht_int64(Z)                                                      # H_m[:, c] diag(D) ...
    return Y * st["du"][:, None]


def modes_apply_int(st: dict, xnum: list) -> list:
    """A x for x = xnum 2^-e (Python integers), as numerators over 2^-(shift_a+e)."""
    m, n = st["m"], st["n"]
    v = [int(st["dv"][j]) * xnum[j] for j in range(n)]
    v = fwht_py(v)
    z = [0] * m
    for k in range(n):
        z[int(st["c"][k])] = int(st["D"][k]) * v[int(st["pi"][k])]
    z = fwht_py(z)
    return [int(st["du"][i]) * z[i] for i in range(m)]


def modes_problem(p: int, m: int = 4096, n: int = 2048, kappa: float = 1e6, seed: int = 0,
                  consistent: bool = True, tag: str = "modes") -> dict:
    """The precision-mode least-squares problem in p limbs.

    A (p, n, m): exact doubles in limb 0 (|A_ij| 2^shift_a < 2^51), zeros
    below.  consistent=True: x* ~ U[-1,1) doubles and b = A x* exactly (at
    most about 130 significant bits, so exact in quad and octo double), so x*
    is the exact least-squares solution.  consistent=False: b ~ U[-1,1) in p
    limbs (the recipe of md_vector); the solution then has the closed form
    V diag(1/sigma) U^T b, which the oracle evaluates from the structure.
    Returns a dict with A, b, xstar (or None) and the structure."""
    st = modes_structure(m, n, kappa, seed, tag)
    Aint = modes_matrix_int(st)
    A = np.zeros((p, n, m), dtype=np.float64)
    A[0] = (Aint.T).astype(np.float64) * 2.0 ** (-st["shift_a"])
    lab = f"{tag}/{m}x{n}/k{kappa:g}/s{seed}/p{p}"
    xstar = None
    if consistent:
        x0 = sym(seed, lab + "/x", n)
        xnum = [int(np.ldexp(v, 53)) for v in x0]          # x = xnum 2^-53 exactly
        bnum = modes_apply_int(st, xnum)
        sh = st["shift_a"] + 53
        b = np.array([split_exact(v, sh, p) for v in bnum]).T.copy()
        xstar = np.zeros((p, n))
        xstar[0] = x0
    else:
        b = md_vector(p, m, seed, lab + "/b")
    return {"A": np.ascontiguousarray(A), "b": np.ascontiguousarray(b), "xstar": xstar, "structure": st}
