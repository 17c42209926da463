"""Lower triangular block-Toeplitz solve on the GPU (one QR of the diagonal
block, then block forward substitution with Algorithm 1 per block) against
the oracle's block forward substitution, every block entrywise and in the
2-norm, with ragged tiles and tall and square blocks."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, assert_close, to_dev, to_host

pytestmark = pytest.mark.gpu


def toe_problem(p, m, n, d1, seed):
    J = np.stack([synth.md_matrix(p, m, n, seed, f"toe/J{i}/{m}x{n}") for i in range(d1)], axis=1)
    b = np.stack([synth.md_vector(p, m, seed, f"toe/b{k}/{m}") for k in range(d1)], axis=1)
    return np.ascontiguousarray(J), np.ascontiguousarray(b)


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,d1,tile", [(12, 9, 4, 4), (40, 30, 5, 8), (100, 64, 6, 32), (64, 64, 3, 64)])
def test_toeplitz_matches_oracle(p, m, n, d1, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    J, b = toe_problem(p, m, n, d1, 17)
    x = torch.zeros((p, d1, n), dtype=torch.float64, device="cuda")
    Jd, bd = to_dev(J), to_dev(b)
    ws = mdls.mdls_toeplitz_lstsq(Jd, bd, x, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    xr = oracle.toeplitz_lstsq(J, b)
    xh = to_host(x)
    for k in range(d1):
        assert_close(np.ascontiguousarray(xh[:, k]), np.ascontiguousarray(xr[:, k]), p, f"block {k}")
    assert np.array_equal(to_host(Jd), J) and np.array_equal(to_host(bd), b)


def test_toeplitz_singular_diagonal_block():
    import torch
    import paper_2110_08375_gb300 as mdls
    p, m, n, d1 = 2, 20, 10, 3
    J, b = toe_problem(p, m, n, d1, 18)
    J[:, 0, 4, :] = 0.0                      # column 4 of J_0 is zero
    x = torch.zeros((p, d1, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_toeplitz_lstsq(to_dev(J), to_dev(b), x, tile=8)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_ERR_SINGULAR
