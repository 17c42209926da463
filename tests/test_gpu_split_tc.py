"""Split mode on the fifth-generation tensor cores (tcgen05): the WY products
of Algorithm 2 (the trailing update C + Y (W^T C), W = -Y T, G = Y^T Y and
the Q accumulation of Section 3) as exact digit products with accumulators
in tensor memory, checked against the oracle's unblocked Householder QR and
least squares with the tolerances of the plain md path, on shapes with
ragged row, column and k tiles, on products whose K range is split over
blocks, and at the full 1024 x 1024, tile-128 size against the cached
oracle answers."""
import os
import sys

import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, assert_close, to_dev, to_host

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_oracle_cache as cache  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture
def engine():
    """Sets the split engine for one test and puts the default back."""
    import paper_2110_08375_gb300 as mdls

    def set_(e):
        mdls.mdls_set_split_engine(e)

    yield set_
    mdls.mdls_set_split_engine(mdls.SPLIT_ENGINE_AUTO)


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", [(130, 70, 32), (200, 129, 32), (300, 260, 64), (160, 150, 128)])
def test_tc_lstsq_matches_oracle(engine, p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    engine(mdls.SPLIT_ENGINE_TCGEN05)
    oracle.set_threads(os.cpu_count() or 1)
    A, b = synth.lstsq_problem(p, m, n, seed=52, tag="split_tc")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=tile, mode=mdls.MODE_SPLIT)
    assert mdls.mdls_read_status(ws) == 0
    assert_close(to_host(xd), oracle.lstsq(A, b), p, f"split tcgen05 lstsq {m}x{n} tile {tile}")


@pytest.mark.parametrize("p", [2, 4, 8])
def test_tc_qr_with_q_matches_oracle(engine, p):
    """400 x 320 at tile 128 (tiles of 128, 128, 64 columns; 400-row products
    over four 128-row tiles, the last one ragged), R and the 400 x 400 Q."""
    import torch
    import paper_2110_08375_gb300 as mdls
    engine(mdls.SPLIT_ENGINE_TCGEN05)
    oracle.set_threads(os.cpu_count() or 1)
    m, n = 400, 320
    A, _ = synth.lstsq_problem(p, m, n, seed=0, tag="qrq")
    Ad = to_dev(A)
    Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_qr(Ad, Qd, tile=128, mode=mdls.MODE_SPLIT)
    assert mdls.mdls_read_status(ws) == 0
    Rr, Qr, _ = oracle.qr(A)
    R, Q = to_host(Ad), to_host(Qd)
    assert_close(R, Rr, p, "R")
    assert_close(Q, Qr, p, "Q")
    for j in range(n):
        assert R[0, j, j] > 0 and np.all(R[:, j, j + 1:] == 0.0)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_tc_agrees_with_mma_sync(engine, p):
    """The two engines compute the same exact digit sums; where the tcgen05
    products split K over blocks (the 128-row products W^T C of a 512 x 384
    problem fill few tiles) the partial products are rounded once more, so
    the factors agree to the md tolerance rather than bit for bit."""
    import torch
    import paper_2110_08375_gb300 as mdls
    m, n = 512, 384
    A, _ = synth.lstsq_problem(p, m, n, seed=3, tag="engines")
    out = {}
    for e in (mdls.SPLIT_ENGINE_MMA_SYNC, mdls.SPLIT_ENGINE_TCGEN05):
        engine(e)
        Ad = to_dev(A)
        Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_qr(Ad, Qd, tile=128, mode=mdls.MODE_SPLIT)
        assert mdls.mdls_read_status(ws) == 0
        out[e] = (to_host(Ad), to_host(Qd))
    (R1, Q1), (R2, Q2) = out[mdls.SPLIT_ENGINE_MMA_SYNC], out[mdls.SPLIT_ENGINE_TCGEN05]
    assert oracle.rel_err(R2, R1) < TOL[p]
    assert oracle.rel_err(Q2, Q1) < TOL[p]


@pytest.mark.parametrize("p", [2, 4, 8])
def test_tc_split_lstsq_n1024_matches_cached_oracle(engine, p):
    """The full dense least-squares size (m = n = 1024, tile 128) in split
    mode with the default engine choice, against the cached oracle answer."""
    import torch
    import paper_2110_08375_gb300 as mdls
    engine(mdls.SPLIT_ENGINE_AUTO)
    entry = cache.load(f"lstsq_n1024_p{p}")
    assert entry is not None, "oracle cache missing: run tests/golden/make_oracle_cache.py cfg1"
    xr, h = entry
    A, b = cache.cfg1_inputs(p)
    assert cache.input_hash(A, b) == h
    xd = torch.zeros((p, 1024), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=128, mode=mdls.MODE_SPLIT)
    assert mdls.mdls_read_status(ws) == 0
    assert_close(to_host(xd), xr, p, "split lstsq n=1024 tile 128")
