"""Writes the cached oracle results that the full-size GPU parity tests read.

Each entry runs only ``oracle/`` (the plain CPU reference) on inputs drawn by
``synth/`` and stores the oracle's answer together with the SHA-256 of the
inputs it was computed from, so that a test can check that it regenerated the
very same inputs before it compares against the cache.

    python tests/golden/make_oracle_cache.py [cfg1] [cfg3] [zls] [--threads N]

cfg1: least squares m = n = 1024 (A and b as drawn for the n = 1024 workload,
      seed 0) in double double, quad double and octo double: x of the
      unblocked Householder QR of [A | b] followed by back substitution.
cfg3: back substitution R x = y in quad double, n = 17920 (diagonal U[1,2],
      strict upper part U[-1,1)/n, y U[-1,1), seed 0).
zls:  complex least squares m = n = 512 (real and imaginary parts of A and b
      drawn as for the dense workload, seed 0) in dd, qd and od; x is stored
      as its real and imaginary parts side by side, (p, 2n).
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CACHE = os.path.join(HERE, "oracle_cache")


def input_hash(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.shape).encode())
        h.update(memoryview(a).cast("B"))
    return h.hexdigest()


def path(name: str) -> str:
    return os.path.join(CACHE, name + ".npz")


def cfg1_inputs(p: int):
    import synth
    return synth.lstsq_problem(p, 1024, 1024, seed=0, tag="cfg1")


def cfg3_inputs():
    import synth
    return synth.upper_triangular_fast(4, 17920, seed=0)


def make_cfg1() -> None:
    import oracle
    for p in (2, 4, 8):
        A, b = cfg1_inputs(p)
        t0 = time.time()
        x = oracle.lstsq(A, b)
        np.savez_compressed(path(f"lstsq_n1024_p{p}"), x=x, input_sha256=input_hash(A, b))
        print(f"cfg1 p={p}: {time.time() - t0:.1f} s", flush=True)


def zls_inputs(p: int):
    import synth
    Ar, br = synth.lstsq_problem(p, 512, 512, seed=0, tag="cplx/ls/re")
    Ai, bi = synth.lstsq_problem(p, 512, 512, seed=0, tag="cplx/ls/im")
    return Ar, Ai, br, bi


def make_zls() -> None:
    import oracle
    for p in (2, 4, 8):
        Ar, Ai, br, bi = zls_inputs(p)
        t0 = time.time()
        xr, xi = oracle.zlstsq(Ar, Ai, br, bi)
        np.savez_compressed(path(f"zlstsq_n512_p{p}"), x=np.concatenate([xr, xi], axis=1),
                            input_sha256=input_hash(Ar, Ai, br, bi))
        print(f"zls p={p}: {time.time() - t0:.1f} s", flush=True)


def make_cfg3() -> None:
    import oracle
    R, y = cfg3_inputs()
    h = input_hash(R, y)
    t0 = time.time()
    x = oracle.backsub(R, y)
    np.savez_compressed(path("backsub_n17920_p4"), x=x, input_sha256=h)
    print(f"cfg3: {time.time() - t0:.1f} s", flush=True)


def load(name: str):
    """(x, input_sha256) of a cached entry, or None when it is absent."""
    f = path(name)
    if not os.path.exists(f):
        return None
    z = np.load(f)
    return z["x"], str(z["input_sha256"])


if __name__ == "__main__":
    import oracle
    args = sys.argv[1:]
    threads = os.cpu_count() or 1
    if "--threads" in args:
        threads = int(args[args.index("--threads") + 1])
    oracle.set_threads(threads)
    os.makedirs(CACHE, exist_ok=True)
    which = [a for a in args if a in ("cfg1", "cfg3", "zls")] or ["cfg1", "cfg3", "zls"]
    if "cfg1" in which:
        make_cfg1()
    if "cfg3" in which:
        make_cfg3()
    if "zls" in which:
        make_zls()
