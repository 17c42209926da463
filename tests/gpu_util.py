"""Helpers shared by the GPU tests: numpy <-> torch marshalling and the error
measures (differences formed exactly by the oracle, then rounded)."""
import numpy as np

TOL = {2: 1e-24, 4: 1e-55, 8: 1e-112}


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def max_entry_err(x, ref) -> float:
    """max_i |x_i - ref_i| / max_i |ref_i| (the difference of each entry is
    formed exactly by the oracle and rounded once): a few bad entries in a
    long vector cannot hide in a 2-norm."""
    import oracle
    d = np.abs(oracle.diff(x, ref))
    scale = float(np.max(np.abs(np.asarray(ref)[0])))
    return float(np.max(d)) / scale if scale else float(np.max(d))


def assert_close(x, ref, p, what=""):
    """Relative 2-norm and entrywise (relative to the largest entry) errors
    both within the tolerance of precision p."""
    import oracle
    e2 = oracle.rel_err(x, ref)
    ei = max_entry_err(x, ref)
    assert e2 < TOL[p] and ei < TOL[p], (what, p, e2, ei)
    return e2, ei
