"""Precision mode "refine" (dd factorisation + iterative refinement in qd/od)
against the oracle: the same tolerances as the plain md solve, an error no
worse than ten times the plain md solve's on an ill-conditioned tall system
(kappa = 1e6, singular values log-spaced from 1 to 1e6), and a failure status
when A is rank deficient at double-double resolution."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = pytest.mark.gpu


def solve(A, b, mode, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    p, n, m = A.shape
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=tile, mode=mode)
    return to_host(xd), mdls.mdls_read_status(ws)


def conditioned(p, m, n, kappa, seed):
    """A = U diag(s) V^T in double (limb 0), U and V orthogonal from numpy's QR
    of seeded normal matrices, s log-spaced 1..kappa; b ~ U[-1,1)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.logspace(0, np.log10(kappa), n)
    Ad = (U * s) @ V.T
    A = np.zeros((p, n, m)); A[0] = Ad.T
    b = synth.md_vector(p, m, seed, "refine/b")
    return A, b


@pytest.mark.parametrize("p", [4, 8])
@pytest.mark.parametrize("m,n,tile", [(256, 256, 32), (200, 129, 32)])
def test_refine_matches_oracle(p, m, n, tile):
    import paper_2110_08375_gb300 as mdls
    A, b = synth.lstsq_problem(p, m, n, seed=12, tag="refine")
    x, st = solve(A, b, mdls.MODE_REFINE, tile)
    assert st == 0, mdls.status_string(st)
    assert oracle.rel_err(x, oracle.lstsq(A, b)) < TOL[p]


@pytest.mark.parametrize("p", [4, 8])
def test_refine_ill_conditioned_matches_plain_accuracy(p):
    import paper_2110_08375_gb300 as mdls
    oracle.set_threads(8)
    A, b = conditioned(p, 192, 96, 1e6, seed=31)
    ref = oracle.lstsq(A, b)
    xr, st = solve(A, b, mdls.MODE_REFINE, 32)
    assert st == 0, mdls.status_string(st)
    xp, st2 = solve(A, b, mdls.MODE_PLAIN, 32)
    assert st2 == 0
    err_ref, err_plain = oracle.rel_err(xr, ref), oracle.rel_err(xp, ref)
    assert err_plain < TOL[p]
    assert err_ref <= 10 * err_plain + TOL[p] * 1e-6, (err_ref, err_plain)


def test_refine_with_dd_is_the_plain_solve():
    import paper_2110_08375_gb300 as mdls
    A, b = synth.lstsq_problem(2, 90, 70, seed=13, tag="refine")
    x1, _ = solve(A, b, mdls.MODE_REFINE, 16)
    x2, _ = solve(A, b, mdls.MODE_PLAIN, 16)
    assert np.array_equal(x1, x2)


def test_refine_reports_failure_when_dd_cannot_resolve_A():
    """Columns 0 and 1 agree in their two leading limbs and differ only in the
    third: rank deficient in double double, full rank in quad double."""
    import paper_2110_08375_gb300 as mdls
    p, m, n = 4, 64, 32
    A, b = synth.lstsq_problem(p, m, n, seed=14, tag="refine")
    A[:, 1, :] = A[:, 0, :]
    A[2, 1, :] = A[1, 1, :] * 2.0 ** -60      # still under half an ulp of limb 1
    A[3, 1, :] = 0.0
    _, st = solve(A, b, mdls.MODE_REFINE, 16)
    assert st in (mdls.MDLS_ERR_NOT_CONVERGED, mdls.MDLS_ERR_SINGULAR)
