"""Precision mode "split": every WY product on the tensor cores as exact
bf16 digit products (error-free splitting), checked against the oracle with
the same tolerances as the plain md path, on tile sizes and shapes with ragged
edges (M, N, K not multiples of the MMA tile), and against the plain path's
accuracy on an ill-conditioned system."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", [(8, 5, 2), (64, 48, 16), (130, 70, 32), (100, 100, 37)])
def test_split_qr_matches_oracle(p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    A, _ = synth.lstsq_problem(p, m, n, seed=41, tag="split")
    Ad = to_dev(A)
    Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_qr(Ad, Qd, tile=tile, mode=mdls.MODE_SPLIT)
    assert mdls.mdls_read_status(ws) == 0
    Rr, Qr, _ = oracle.qr(A)
    R = to_host(Ad)
    assert oracle.rel_err(R, Rr) < TOL[p]
    assert oracle.rel_err(to_host(Qd), Qr) < TOL[p]
    for j in range(n):
        assert R[0, j, j] > 0 and np.all(R[:, j, j + 1:] == 0.0)


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", [(10, 7, 3), (200, 129, 32), (256, 256, 32)])
def test_split_lstsq_matches_oracle(p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    oracle.set_threads(8)
    A, b = synth.lstsq_problem(p, m, n, seed=42, tag="split")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=tile, mode=mdls.MODE_SPLIT)
    assert mdls.mdls_read_status(ws) == 0
    assert oracle.rel_err(to_host(xd), oracle.lstsq(A, b)) < TOL[p]


def test_split_upper_triangular_is_exact():
    import torch
    import paper_2110_08375_gb300 as mdls
    p, m, n = 4, 40, 33
    rng = np.random.default_rng(5)
    U = np.zeros((p, n, m))
    for j in range(n):
        U[0, j, :j] = rng.integers(-5, 5, j)
        U[0, j, j] = rng.integers(1, 5)
    Ad = to_dev(U)
    Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    mdls.mdls_qr(Ad, Qd, tile=8, mode=mdls.MODE_SPLIT)
    assert np.array_equal(to_host(Ad), U)
    assert np.array_equal(to_host(Qd)[0], np.eye(m)) and not to_host(Qd)[1:].any()


@pytest.mark.parametrize("p", [4, 8])
def test_split_ill_conditioned_matches_plain_accuracy(p):
    import torch
    import paper_2110_08375_gb300 as mdls
    from test_gpu_refine import conditioned
    oracle.set_threads(8)
    A, b = conditioned(p, 192, 96, 1e6, seed=33)
    ref = oracle.lstsq(A, b)
    errs = {}
    for mode in (mdls.MODE_PLAIN, mdls.MODE_SPLIT):
        xd = torch.zeros((p, 96), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=32, mode=mode)
        assert mdls.mdls_read_status(ws) == 0
        errs[mode] = oracle.rel_err(to_host(xd), ref)
    assert errs[mdls.MODE_PLAIN] < TOL[p]
    assert errs[mdls.MODE_SPLIT] <= 10 * errs[mdls.MODE_PLAIN] + TOL[p] * 1e-6, errs
