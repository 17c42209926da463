"""Parity at the full size of the dense least-squares workload: m = n = 1024,
tile 128 (eight tiles, so the tile-128 look-ahead, the wave-aware split-K
choices of the 1024-row products and the octo-double 16 x 8 product grids all
run), in double double, quad double and octo double, against the oracle's
unblocked Householder least squares (Section 1, Algorithm 2 then Algorithm 1
of arXiv 2110.08375).  The oracle's answers at this size take minutes, so they
are cached under tests/golden/oracle_cache/ by make_oracle_cache.py (which
calls only the oracle) together with the SHA-256 of the inputs they were
computed from; the test regenerates the inputs and checks that hash first.

Also the QR with Q formed (Algorithm 2's full output) on a multi-tile
tile-128 problem with a ragged last tile, R and Q against the oracle."""
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


@pytest.mark.parametrize("p", [2, 4, 8])
def test_lstsq_n1024_tile128_matches_cached_oracle(p):
    import torch
    import paper_2110_08375_gb300 as mdls
    entry = cache.load(f"lstsq_n1024_p{p}")
    assert entry is not None, "oracle cache missing: run tests/golden/make_oracle_cache.py cfg1"
    xr, h = entry
    A, b = cache.cfg1_inputs(p)
    assert cache.input_hash(A, b) == h, "inputs differ from those the cache was computed from"
    Ad, bd = to_dev(A), to_dev(b)
    xd = torch.zeros((p, 1024), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(Ad, bd, xd, tile=128)
    assert mdls.mdls_read_status(ws) == 0
    assert_close(to_host(xd), xr, p, "lstsq n=1024 tile 128")
    # a second call on the same workspace (as the benchmark's timed steps run
    # it) gives the same bits
    x2 = torch.zeros_like(xd)
    mdls.mdls_lstsq(Ad, bd, x2, tile=128, ws=ws)
    assert mdls.mdls_read_status(ws) == 0
    assert torch.equal(xd, x2)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_qr_with_q_multitile_tile128(p):
    """m = 400, n = 320 at tile 128: tiles of 128, 128 and 64 columns, the
    look-ahead panel, and the backward accumulation of the 400 x 400 Q."""
    import torch
    import paper_2110_08375_gb300 as mdls
    oracle.set_threads(os.cpu_count() or 1)
    m, n = 400, 320
    A, _ = synth.lstsq_problem(p, m, n, seed=0, tag="qrq")
    Ad = to_dev(A)
    Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_qr(Ad, Qd, tile=128)
    assert mdls.mdls_read_status(ws) == 0
    Rr, Qr, _ = oracle.qr(A)
    R, Q = to_host(Ad), to_host(Qd)
    assert_close(R, Rr, p, "R")
    assert_close(Q, Qr, p, "Q")
    for j in range(n):
        assert R[0, j, j] > 0 and np.all(R[:, j, j + 1:] == 0.0)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_zlstsq_n512_tile128_matches_cached_oracle(p):
    """Complex least squares at the size of the paper's complex QR study
    (512 x 512), tile 128, against the complex oracle's cached answer."""
    import torch
    import paper_2110_08375_gb300 as mdls
    entry = cache.load(f"zlstsq_n512_p{p}")
    assert entry is not None, "oracle cache missing: run tests/golden/make_oracle_cache.py zls"
    xref, h = entry
    Ar, Ai, br, bi = cache.zls_inputs(p)
    assert cache.input_hash(Ar, Ai, br, bi) == h
    n = 512
    xr = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    xi = torch.zeros_like(xr)
    ws = mdls.mdls_zlstsq(to_dev(Ar), to_dev(Ai), to_dev(br), to_dev(bi), xr, xi, tile=128)
    assert mdls.mdls_read_status(ws) == 0
    got = np.concatenate([to_host(xr), to_host(xi)], axis=1)
    assert_close(got, xref, p, "zlstsq n=512 tile 128")
