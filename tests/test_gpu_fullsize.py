"""Full-size workloads, checked with O(n) or O(mn) oracle work:

* back substitution, quad double, n = 17920, tile 128 (140 tiles), diagonal
  U[1,2], strict upper U[-1,1]/n, y U[-1,1): the last tile of x depends only
  on the trailing block of R and y, so the oracle solves that block exactly;
  48 sampled rows of the residual y - R x are formed by the oracle;
* precision modes at m = 4096, n = 2048, tile 128, A = U diag(s) V^T with
  s log-spaced from 1 to 1e6, qd and od: the oracle forms A^T (b - A x) for
  the split and refine solutions, and the two solutions agree.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_backsub_qd_17920():
    import torch
    import paper_2110_08375_gb300 as mdls
    p, n, t = 4, 17920, 128
    R, y = synth.upper_triangular_fast(p, n, seed=0)
    Rd = torch.from_numpy(R).cuda()
    yd = to_dev(y)
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_backsub(Rd, yd, xd, tile=t)
    assert mdls.mdls_read_status(ws) == 0
    x = to_host(xd)
    del Rd
    # the trailing tile exactly
    o = n - t
    Rt = np.ascontiguousarray(R[:, o:, o:])
    xt = oracle.backsub(Rt, np.ascontiguousarray(y[:, o:]))
    assert oracle.rel_err(x[:, o:], xt) < TOL[p]
    # sampled residual rows r_i = y_i - sum_j R_ij x_j, relative to |y| + |R||x|
    rng = np.random.default_rng(1)
    for i in sorted(rng.choice(n, 48, replace=False)):
        k = n - i
        Arow = np.zeros((p, k, 1))
        Arow[:, :, 0] = R[:, i:, i]
        Ax = oracle.gemv(Arow, np.ascontiguousarray(x[:, i:]))
        r = oracle.diff(y[:, i:i + 1], Ax)[0]
        scale = abs(y[0, i]) + np.sum(np.abs(R[0, i:, i]) * np.abs(x[0, i:]))
        assert abs(r) <= 1e-58 * scale, (i, r, scale)


@pytest.mark.parametrize("p", [4, 8])
def test_modes_4096x2048(p):
    import torch
    import paper_2110_08375_gb300 as mdls
    from test_gpu_refine import conditioned
    oracle.set_threads(16)
    m, n, t = 4096, 2048, 128
    A, b = conditioned(p, m, n, 1e6, seed=2)
    Ad, bd = to_dev(A), to_dev(b)
    xs = {}
    for mode in (mdls.MODE_SPLIT, mdls.MODE_REFINE):
        xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_lstsq(Ad, bd, xd, tile=t, mode=mode)
        assert mdls.mdls_read_status(ws) == 0
        xs[mode] = to_host(xd)
        del ws
    normA = np.sqrt(np.sum(A[0] ** 2))
    for mode, x in xs.items():
        r = oracle.residual(A, x, b)
        g = oracle.gemv(A, r, trans=True)                 # A^T (b - A x)
        rel = np.linalg.norm(g[0]) / (normA * np.linalg.norm(r[0]))
        assert rel < (1e-58 if p == 4 else 1e-120), (mode, rel)
    # the two modes agree to kappa times the unit roundoff
    assert oracle.rel_err(xs[mdls.MODE_SPLIT], xs[mdls.MODE_REFINE]) < (1e-55 if p == 4 else 1e-112)
