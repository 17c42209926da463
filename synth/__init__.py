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
