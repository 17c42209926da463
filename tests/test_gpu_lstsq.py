"""Least squares (QR of [A | b], then Algorithm 1) and back substitution on
the GPU against the oracle, elementwise within the stated tolerances, plus the
device status of a singular system."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, assert_close, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("m,n,tile", [(10, 7, 3), (64, 48, 16), (200, 129, 32), (128, 128, 128)])
def test_lstsq_matches_oracle(p, m, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    A, b = synth.lstsq_problem(p, m, n, seed=7, tag="lstest")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    Ad, bd = to_dev(A), to_dev(b)
    ws = mdls.mdls_lstsq(Ad, bd, xd, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    assert oracle.rel_err(to_host(xd), oracle.lstsq(A, b)) < TOL[p]
    # inputs are read only
    assert np.array_equal(to_host(Ad), A) and np.array_equal(to_host(bd), b)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_lstsq_small_config_full_size(p):
    """n = 256, tile 32 (eight tiles): the smallest benchmark configuration,
    run here in every precision."""
    import torch
    import paper_2110_08375_gb300 as mdls
    oracle.set_threads(8)
    n = 256
    A, b = synth.lstsq_problem(p, n, n, seed=0, tag="cfg0")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=32)
    assert mdls.mdls_read_status(ws) == 0
    assert oracle.rel_err(to_host(xd), oracle.lstsq(A, b)) < TOL[p]


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("n,tile", [(1, 1), (5, 2), (64, 16), (100, 32), (257, 64), (300, 256)])
def test_backsub_matches_oracle(p, n, tile):
    import torch
    import paper_2110_08375_gb300 as mdls
    R, y = synth.upper_triangular(p, n, seed=3)
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_backsub(to_dev(R), to_dev(y), xd, tile=tile)
    assert mdls.mdls_read_status(ws) == 0
    assert oracle.rel_err(to_host(xd), oracle.backsub(R, y)) < TOL[p]


def test_backsub_singular_status():
    import torch
    import paper_2110_08375_gb300 as mdls
    p, n = 2, 40
    R, y = synth.upper_triangular(p, n, seed=4)
    R[:, 17, 17] = 0.0
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_backsub(to_dev(R), to_dev(y), xd, tile=16)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_ERR_SINGULAR


def test_workspace_reuse_gives_identical_results():
    """Deterministic: the same call twice on one workspace is bitwise equal."""
    import torch
    import paper_2110_08375_gb300 as mdls
    p, m, n = 4, 90, 70
    A, b = synth.lstsq_problem(p, m, n, seed=8, tag="det")
    Ad, bd = to_dev(A), to_dev(b)
    x1 = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(x1)
    ws = mdls.mdls_lstsq(Ad, bd, x1, tile=16)
    mdls.mdls_lstsq(Ad, bd, x2, tile=16, ws=ws)
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_lstsq_widest_tile(p):
    """Tile 256, the widest the ABI accepts: the panel's 256 column blocks must
    all be resident at once (cooperative launch), in every precision."""
    import torch
    import paper_2110_08375_gb300 as mdls
    m, n = 300, 260
    A, b = synth.lstsq_problem(p, m, n, seed=9, tag="wide")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=256)
    assert mdls.mdls_read_status(ws) == 0
    assert oracle.rel_err(to_host(xd), oracle.lstsq(A, b)) < TOL[p]


@pytest.fixture
def schedule():
    """Sets the back substitution's step-2 schedule for one test and restores
    the automatic choice afterwards."""
    import paper_2110_08375_gb300 as mdls
    yield mdls.mdls_set_backsub_schedule
    mdls.mdls_set_backsub_schedule(mdls.BS_AUTO)


@pytest.mark.parametrize("p", [2, 4, 8])
@pytest.mark.parametrize("n,tile", [(32, 32), (33, 32), (100, 32), (257, 64), (300, 64), (1000, 128),
                                    (700, 256)])
def test_backsub_persistent_schedule_matches_oracle(p, n, tile, schedule):
    """The persistent launch of step 2 (bulk updates from a task queue, the
    chain x_i -> x_{i-1} on reserved SMs) against the oracle, with ragged
    last tiles and one-tile problems; the per-step schedule on the same
    input agrees with it."""
    import torch
    import paper_2110_08375_gb300 as mdls
    R, y = synth.upper_triangular(p, n, seed=13)
    Rd, yd = to_dev(R), to_dev(y)
    xs = {}
    for sch in (mdls.BS_PERSISTENT, mdls.BS_PER_STEP):
        schedule(sch)
        xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_backsub(Rd, yd, xd, tile=tile)
        assert mdls.mdls_read_status(ws) == 0
        xs[sch] = to_host(xd)
    xr = oracle.backsub(R, y)
    assert_close(xs[mdls.BS_PERSISTENT], xr, p, "persistent")
    assert_close(xs[mdls.BS_PER_STEP], xr, p, "per step")


@pytest.mark.parametrize("p", [2, 4, 8])
def test_lstsq_with_persistent_back_substitution(p, schedule):
    import torch
    import paper_2110_08375_gb300 as mdls
    schedule(mdls.BS_PERSISTENT)
    m, n = 230, 200
    A, b = synth.lstsq_problem(p, m, n, seed=14, tag="lspersist")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=32)
    assert mdls.mdls_read_status(ws) == 0
    assert_close(to_host(xd), oracle.lstsq(A, b), p, "lstsq persistent")


def test_backsub_persistent_singular_status(schedule):
    import torch
    import paper_2110_08375_gb300 as mdls
    schedule(mdls.BS_PERSISTENT)
    p, n = 4, 200
    R, y = synth.upper_triangular(p, n, seed=15)
    R[:, 150, 150] = 0.0
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    ws = mdls.mdls_backsub(to_dev(R), to_dev(y), xd, tile=32)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_ERR_SINGULAR
