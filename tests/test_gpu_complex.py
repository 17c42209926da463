"""Complex multiple-double QR, back substitution and least squares on the GPU
(the paper's algorithms on complex data: Hermitian transposes, real and
imaginary parts kept separately) against the complex oracle, entrywise and in
the 2-norm, with ragged last tiles, one-tile problems, tall and square
shapes; the zero-pivot status; real data through the complex path."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, max_entry_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def zproblem(p, m, n, seed, tag):
    Ar, br = synth.lstsq_problem(p, m, n, seed=seed, tag=tag + "/re")
    Ai, bi = synth.lstsq_problem(p, m, n, seed=seed, tag=tag + "/im")
    return Ar, Ai, br, bi


def zclose(xr, xi, rr, ri, p, what=""):
    e2 = oracle.zrel_err(xr, xi, rr, ri)
    scale = max(np.max(np.abs(rr[0])), np.max(np.abs(ri[0])))
    ei = max(np.max(np.abs(oracle.diff(xr, rr))), np.max(np.abs(oracle.diff(xi, ri)))) / scale
    assert e2 < TOL[p] and ei < TOL[p], (what, p, e2, ei)


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", [(10, 7, 3), (64, 48, 16), (130, 100, 32), (96, 96, 96)])
def test_zlstsq_matches_oracle(p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    oracle.set_threads(8)
    Ar, Ai, br, bi = zproblem(p, m, n, 3, "zls")
    xr = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    xi = torch.zeros_like(xr)
    dA = [to_dev(Ar), to_dev(Ai)]
    ws = mdls.mdls_zlstsq(dA[0], dA[1], to_dev(br), to_dev(bi), xr, xi, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    rr, ri = oracle.zlstsq(Ar, Ai, br, bi)
    zclose(to_host(xr), to_host(xi), rr, ri, p, "zlstsq")
    assert np.array_equal(to_host(dA[0]), Ar) and np.array_equal(to_host(dA[1]), Ai)


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", [(9, 6, 2), (40, 30, 8), (100, 70, 32)])
def test_zqr_with_q_matches_oracle(p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    Ar, Ai, _, _ = zproblem(p, m, n, 4, "zqr")
    dAr, dAi = to_dev(Ar), to_dev(Ai)
    Qr = torch.zeros((p, m, m), dtype=torch.float64, device="cuda")
    Qi = torch.zeros_like(Qr)
    ws = mdls.mdls_zqr(dAr, dAi, Qr, Qi, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    Rr, Ri, QRr, QRi, _ = oracle.zqr(Ar, Ai)
    zclose(to_host(dAr), to_host(dAi), Rr, Ri, p, "R")
    zclose(to_host(Qr), to_host(Qi), QRr, QRi, p, "Q")
    R = to_host(dAr)
    for j in range(n):
        assert np.all(R[:, j, j + 1:] == 0.0) and np.all(to_host(dAi)[:, j, j + 1:] == 0.0)


def zupper(p, n, seed):
    Rr, yr = synth.upper_triangular(p, n, seed=seed, tag="zbs/re")
    Ri, yi = synth.upper_triangular(p, n, seed=seed, tag="zbs/im")
    return Rr, Ri, yr, yi


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("n,tile", [(1, 1), (5, 2), (64, 16), (100, 32), (257, 64)])
def test_zbacksub_matches_oracle(p, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    Rr, Ri, yr, yi = zupper(p, n, 5)
    xr = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    xi = torch.zeros_like(xr)
    ws = mdls.mdls_zbacksub(to_dev(Rr), to_dev(Ri), to_dev(yr), to_dev(yi), xr, xi, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    rr, ri = oracle.zbacksub(Rr, Ri, yr, yi)
    zclose(to_host(xr), to_host(xi), rr, ri, p, "zbacksub")


def test_zbacksub_singular_status():
    import torch
    import paper_2110_08375_gb300 as mdls
    p, n = 2, 40
    Rr, Ri, yr, yi = zupper(p, n, 6)
    Rr[:, 17, 17] = 0.0
    Ri[:, 17, 17] = 0.0
    xr = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    xi = torch.zeros_like(xr)
    ws = mdls.mdls_zbacksub(to_dev(Rr), to_dev(Ri), to_dev(yr), to_dev(yi), xr, xi, tile=16)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_ERR_SINGULAR


@pytest.mark.parametrize("p", [2, 4])
def test_real_data_through_the_complex_path(p):
    """Zero imaginary parts stay exactly zero and the real part is the real
    least-squares solution."""
    import torch
    import paper_2110_08375_gb300 as mdls
    m, n = 70, 50
    A, b = synth.lstsq_problem(p, m, n, seed=7, tag="zrealdata")
    z, zb = np.zeros_like(A), np.zeros_like(b)
    xr = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    xi = torch.zeros_like(xr)
    ws = mdls.mdls_zlstsq(to_dev(A), to_dev(z), to_dev(b), to_dev(zb), xr, xi, tile=16)
    assert mdls.mdls_read_status(ws) == 0
    assert np.all(to_host(xi) == 0.0)
    assert oracle.rel_err(to_host(xr), oracle.lstsq(A, b)) < TOL[p]
