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
