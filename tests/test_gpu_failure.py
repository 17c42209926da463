"""Failure detection without a GPU fault: every device wait of the library is
bounded.  The Householder panel runs the columns of a tile in separate blocks
that wait on flags published by the blocks before them (Section 3: the
columns of a tile are reduced one after another); if a flag never came, the
wait gives up after its limit, records MDLS_ERR_TIMEOUT in the workspace
status and returns.  mdls_wait_check runs that same wait on a flag nothing
publishes, with a short limit; the status must read MDLS_ERR_TIMEOUT and the
GPU must still run a solve correctly afterwards."""
import pytest

import oracle
import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_gpu_stays_usable():
    import torch
    import paper_2110_08375_gb300 as mdls
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ws = mdls.mdls_wait_check(2_000_000, publish=False)       # 2 ms limit, flag never set
    e1.record(stream)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_ERR_TIMEOUT
    waited = e0.elapsed_time(e1)
    assert 1.9 <= waited < 1000.0, waited                    # gave up after its limit, not before
    # the same wait with the flag published ends normally
    ws2 = mdls.mdls_wait_check(1_000_000_000, publish=True)
    assert mdls.mdls_read_status(ws2) == mdls.MDLS_OK
    # and the context still solves a problem correctly
    p, m, n = 4, 70, 50
    A, b = synth.lstsq_problem(p, m, n, seed=31, tag="after-timeout")
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    wsl = mdls.mdls_lstsq(to_dev(A), to_dev(b), xd, tile=16)
    assert mdls.mdls_read_status(wsl) == mdls.MDLS_OK
    assert oracle.rel_err(to_host(xd), oracle.lstsq(A, b)) < TOL[p]


def test_status_of_a_new_call_starts_clean_after_a_timeout():
    """A workspace whose header recorded a timeout is cleared by the next
    call that uses it."""
    import torch
    import paper_2110_08375_gb300 as mdls
    p, n = 2, 64
    R, y = synth.upper_triangular(p, n, seed=32)
    need = max(mdls.mdls_backsub_workspace(p, n, 16), mdls.WAIT_CHECK_WORKSPACE)
    ws = mdls.workspace(need)
    mdls.mdls_wait_check(1_000_000, publish=False, ws=ws)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_ERR_TIMEOUT
    xd = torch.zeros((p, n), dtype=torch.float64, device="cuda")
    mdls.mdls_backsub(to_dev(R), to_dev(y), xd, tile=16, ws=ws)
    assert mdls.mdls_read_status(ws) == mdls.MDLS_OK
    assert oracle.rel_err(to_host(xd), oracle.backsub(R, y)) < TOL[p]
