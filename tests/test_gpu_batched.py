"""Batched least squares: mixed shapes and precisions in one graph launch,
each solution checked against the oracle; explicit and autotuned tiles and
modes; a replay gives identical bits; invalid problems are rejected at
planning."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = pytest.mark.gpu


def make(shapes, seed=3):
    import torch
    probs, host = [], []
    for idx, (m, n, p) in enumerate(shapes):
        A, b = synth.batched_problem(idx, m, n, p, seed=seed)
        x = torch.zeros((p, n), dtype=torch.float64, device="cuda")
        probs.append((to_dev(A), to_dev(b), x))
        host.append((A, b))
    return probs, host


def test_batched_matches_oracle():
    import paper_2110_08375_gb300 as mdls
    shapes = synth.batched_shapes(24, seed=7, nmin=8, nmax=96)
    probs, host = make(shapes)
    plan = mdls.mdls_batched_plan(probs, autotune=True)
    plan.launch()
    assert plan.status() == [0] * len(shapes)
    for (A, b), (_, _, x), (m, n, p) in zip(host, probs, shapes):
        assert oracle.rel_err(to_host(x), oracle.lstsq(A, b)) < TOL[p], (m, n, p)
    tiles = plan.tiles()
    assert all(1 <= t <= n for t, (m, n, p) in zip(tiles, shapes))
    assert set(plan.modes()) <= {mdls.MODE_PLAIN, mdls.MODE_SPLIT}
    # a replay is bitwise identical
    first = [to_host(x).copy() for (_, _, x) in probs]
    for (_, _, x) in probs:
        x.zero_()
    plan.launch()
    assert all(np.array_equal(f, to_host(x)) for f, (_, _, x) in zip(first, probs))
    plan.destroy()


def test_batched_explicit_tiles_and_single_solve_agree():
    import torch
    import paper_2110_08375_gb300 as mdls
    shapes = [(40, 33, 2), (70, 64, 4), (12, 12, 8)]
    probs, host = make(shapes, seed=4)
    plan = mdls.mdls_batched_plan([(A, b, x, 8) for (A, b, x) in probs], autotune=False)
    assert plan.tiles() == [8, 8, 8]
    plan.launch()
    assert plan.status() == [0, 0, 0]
    for (A, b, x), (m, n, p) in zip(probs, shapes):
        xs = torch.zeros_like(x)
        mdls.mdls_lstsq(A, b, xs, tile=8)
        assert oracle.rel_err(to_host(x), to_host(xs)) < TOL[p]


def test_batched_rejects_invalid_problem():
    import torch
    import paper_2110_08375_gb300 as mdls
    A = torch.zeros((2, 5, 4), dtype=torch.float64, device="cuda")     # m = 4 < n = 5
    b = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    x = torch.zeros((2, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(mdls.MdlsError):
        mdls.mdls_batched_plan([(A, b, x)])


def test_lstsq_batched_device_array_and_status():
    """mdls_lstsq_batched: the problem array and the per-problem status on the
    device, one call; every solution against the oracle; a zero column makes
    exactly that problem's status MDLS_ERR_SINGULAR; a second call (served by
    the cached plan) gives the same bits."""
    import torch
    import paper_2110_08375_gb300 as mdls
    shapes = synth.batched_shapes(24, seed=11, nmin=8, nmax=96)
    probs, host = make(shapes, seed=5)
    bad = 5
    probs[bad][0][:, 2, :] = 0.0                       # column 2 of problem 5 is zero
    host[bad] = (to_host(probs[bad][0]), host[bad][1])
    probs_dev = mdls.problems_device(probs)
    ws, status = mdls.mdls_lstsq_batched(probs, probs_dev=probs_dev)
    torch.cuda.synchronize()
    st = status.cpu().tolist()
    assert st[bad] == mdls.MDLS_ERR_SINGULAR
    assert all(s == 0 for i, s in enumerate(st) if i != bad)
    for i, ((A, b), (_, _, x), (m, n, p)) in enumerate(zip(host, probs, shapes)):
        if i != bad:
            assert oracle.rel_err(to_host(x), oracle.lstsq(A, b)) < TOL[p], (i, m, n, p)
    first = [to_host(x).copy() for (_, _, x) in probs]
    for (_, _, x) in probs:
        x.zero_()
    status.fill_(-99)
    mdls.mdls_lstsq_batched(probs, ws=ws, status=status, probs_dev=probs_dev)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == st
    assert all(np.array_equal(f, to_host(x)) for i, (f, (_, _, x)) in enumerate(zip(first, probs)) if i != bad)


def test_lstsq_batched_rejects_invalid_problem_before_launch():
    import torch
    import paper_2110_08375_gb300 as mdls
    A = torch.zeros((2, 5, 4), dtype=torch.float64, device="cuda")     # m = 4 < n = 5
    b = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    x = torch.zeros((2, 5), dtype=torch.float64, device="cuda")
    probs_dev = mdls.problems_device([(A, b, x)])
    L = mdls.lib()
    assert L.mdls_lstsq_batched_workspace(probs_dev.data_ptr(), 1) == 0
    ws = mdls.workspace(1 << 20)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = L.mdls_lstsq_batched(probs_dev.data_ptr(), 1, ws.data_ptr(), 1 << 20, st.data_ptr(), None)
    assert rc == mdls.MDLS_ERR_ARG
