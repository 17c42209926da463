"""Blocked Householder QR (Algorithm 2) on the GPU against the oracle's
unblocked QR: R and Q elementwise within the stated relative-norm
tolerances, on several tile sizes, ragged last tiles, tall and square shapes
(arXiv 2110.08375, Section 3)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = pytest.mark.gpu

SHAPES = [(8, 5, 2), (33, 17, 8), (64, 64, 16), (100, 37, 16), (130, 70, 32), (96, 96, 96)]


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", SHAPES)
def test_qr_matches_oracle(p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    A, _ = synth.lstsq_problem(p, m, n, seed=5, tag="qrtest")
    Ad = to_dev(A)
    Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_qr(Ad, Qd, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    R = to_host(Ad)
    Q = to_host(Qd)
    Rr, Qr, _ = oracle.qr(A)
    assert oracle.rel_err(R, Rr) < TOL[p]
    assert oracle.rel_err(Q, Qr) < TOL[p]
    for j in range(n):
        assert R[0, j, j] > 0
        assert np.all(R[:, j, j + 1:] == 0.0)


@pytest.mark.parametrize("p", [2, 4])
def test_qr_without_q_matches(p):
    import paper_2110_08375_gb300 as mdls
    m, n, tile = 77, 60, 16
    A, _ = synth.lstsq_problem(p, m, n, seed=6, tag="qrtest")
    Ad = to_dev(A)
    ws = mdls.mdls_qr(Ad, None, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    Rr, _, _ = oracle.qr(A, want_q=False)
    assert oracle.rel_err(to_host(Ad), Rr) < TOL[p]


def test_qr_special_cases_exact():
    """Upper triangular input with positive diagonal: every reflector is the
    identity, so R = A and Q = I exactly; a diagonal with negative entries
    flips signs exactly."""
    import torch
    import paper_2110_08375_gb300 as mdls
    p, m, n = 2, 12, 9
    U = np.zeros((p, n, m))
    rng = np.random.default_rng(0)
    for j in range(n):
        U[0, j, :j] = rng.integers(-5, 5, j)
        U[0, j, j] = rng.integers(1, 5)
    Ad = to_dev(U)
    Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    mdls.mdls_qr(Ad, Qd, tile=4)
    assert np.array_equal(to_host(Ad), U)
    assert np.array_equal(to_host(Qd)[0], np.eye(m)) and not to_host(Qd)[1].any()
    D = np.zeros((p, 3, 3)); D[0] = np.diag([-3.0, 2.0, -0.5])
    Ad = to_dev(D)
    Qd = torch.zeros((p, 3, 3), dtype=torch.float64, device="cuda")
    mdls.mdls_qr(Ad, Qd, tile=2)
    assert np.array_equal(to_host(Ad)[0], np.diag([3.0, 2.0, 0.5]))
    assert np.array_equal(to_host(Qd)[0], np.diag([-1.0, 1.0, -1.0]))


@pytest.mark.parametrize("p", [2, 8])
def test_tall_skinny_uses_split_k(p):
    """A tall, narrow QR: every product has a small output grid and a long K,
    so the GEMMs run split-K (partials summed in a fixed order); R and Q must
    still match the oracle, and two runs must agree bitwise."""
    import torch
    import paper_2110_08375_gb300 as mdls
    m, n, tile = 700, 24, 8
    A, _ = synth.lstsq_problem(p, m, n, seed=9, tag="qrtest")
    outs = []
    for _ in range(2):
        Ad = to_dev(A)
        Qd = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_qr(Ad, Qd, tile=tile)
        assert mdls.mdls_read_status(ws) == 0
        outs.append((to_host(Ad), to_host(Qd)))
    Rr, Qr, _ = oracle.qr(A)
    assert oracle.rel_err(outs[0][0], Rr) < TOL[p]
    assert oracle.rel_err(outs[0][1], Qr) < TOL[p]
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
