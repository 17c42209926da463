"""Full-size workloads:

* back substitution, quad double, n = 17920, tile 128 (140 tiles), diagonal
  U[1,2], strict upper U[-1,1]/n, y U[-1,1): the whole x against the cached
  oracle solution of the same inputs;
* precision modes at m = 4096, n = 2048, tile 128, A = U diag(sigma) V^T
  with exactly orthogonal Walsh-Hadamard factors and sigma log-spaced over a
  condition number of 1e6, qd and od: every mode against the exact solution.
"""
import os
import sys

import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, assert_close, max_entry_err, to_dev, to_host

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_oracle_cache as cache  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_backsub_qd_17920():
    """The whole x against the oracle's row-by-row back substitution of the
    same R and y (cached with the SHA-256 of the inputs), entrywise and in
    the 2-norm, at the tile and launch configuration the benchmark times."""
    import torch
    import paper_2110_08375_gb300 as mdls
    entry = cache.load("backsub_n17920_p4")
    assert entry is not None, "oracle cache missing: run tests/golden/make_oracle_cache.py cfg3"
    xr, h = entry
    p, n, t = 4, 17920, 128
    R, y = cache.cfg3_inputs()
    assert cache.input_hash(R, y) == h, "inputs differ from those the cache was computed from"
    Rd = torch.from_numpy(R).cuda()
    del R
    yd = to_dev(y)
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_backsub(Rd, yd, xd, tile=t)
    assert mdls.mdls_read_status(ws) == 0
    assert_close(to_host(xd), xr, p, "backsub qd n=17920 tile 128")
    # tile 64 as well (280 tiles)
    x2 = torch.zeros_like(xd)
    ws2 = mdls.mdls_backsub(Rd, yd, x2, tile=64)
    assert mdls.mdls_read_status(ws2) == 0
    assert_close(to_host(x2), xr, p, "backsub qd n=17920 tile 64")


@pytest.mark.parametrize("p", [4, 8])
@pytest.mark.parametrize("consistent", [True, False])
def test_modes_4096x2048_against_closed_form(p, consistent):
    """Precision modes at m = 4096, n = 2048, tile 128, kappa = 1e6: plain md
    QR, split products on the tensor cores and dd factorisation with
    refinement, each compared with the exact least-squares solution (x* drawn
    and b = A x* formed exactly, or b drawn and x* = V diag(1/sigma) U^T b from
    the oracle's closed form).  "Equal stated accuracy": each mode's error is
    at most 10 times the plain md error (or below the plain tolerance)."""
    import torch
    import paper_2110_08375_gb300 as mdls
    from oracle import closed_form
    m, n, t = 4096, 2048, 128
    pr = synth.modes_problem(p, m, n, 1e6, seed=0, consistent=consistent)
    xstar = pr["xstar"] if consistent else closed_form.modes_solution(pr["structure"], pr["b"], p)
    Ad, bd = to_dev(pr["A"]), to_dev(pr["b"])
    errs = {}
    for name, mode in (("plain", mdls.MODE_PLAIN), ("split", mdls.MODE_SPLIT), ("refine", mdls.MODE_REFINE)):
        xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_lstsq(Ad, bd, xd, tile=t, mode=mode)
        assert mdls.mdls_read_status(ws) == 0, name
        del ws
        x = to_host(xd)
        errs[name] = (oracle.rel_err(x, xstar), max_entry_err(x, xstar))
    print(f"p={p} consistent={consistent} errors vs x*:", errs)
    plain = errs["plain"][0]
    # kappa u_p n bounds the forward error of a consistent system; an
    # inconsistent one adds kappa^2 u_p ||r|| / (||A|| ||x||)
    bound = (1e6 if consistent else 1e12) * n * 2.0 ** (-53 * p)
    assert plain < bound, errs
    for name in ("split", "refine"):
        assert errs[name][0] <= max(10 * plain, TOL[p]), (name, errs)
