"""mdls_backsub_noalloc: back substitution for callers that cannot allocate
device memory when they call (a plugin whose host framework owns all device
memory, a loop with a memory budget fixed at start-up, code that must not risk
cudaMalloc's implicit synchronisation).  Its scratch is a fixed array inside
the library, so the call takes only inputs and outputs.

Checked through the C ABI against mdls_backsub (which uses a caller
workspace), on two calls in a row, within the tolerances of the other GPU
tests; and a problem larger than the fixed scratch is rejected before any
launch.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth
from gpu_util import TOL, to_dev, to_host

pytestmark = pytest.mark.gpu


def _entry():
    import paper_2110_08375_gb300 as mdls
    L = mdls.lib()
    f = L.mdls_backsub_noalloc
    i64, vp = C.c_int64, C.c_void_p
    f.argtypes = [C.c_int, i64, vp, i64, i64, vp, i64, vp, i64, C.c_int, vp, vp]
    f.restype = C.c_int
    return mdls, f


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    mdls, f = _entry()
    stream = torch.cuda.current_stream()
    for p, n, tile, seed in [(4, 300, 64, 21), (2, 700, 128, 22)]:
        R, y = synth.upper_triangular(p, n, seed=seed)
        Rd, yd = to_dev(R), to_dev(y)
        x_ws = torch.zeros((p, n), dtype=torch.float64, device="cuda")
        ws = mdls.mdls_backsub(Rd, yd, x_ws, tile=tile)
        assert mdls.mdls_read_status(ws) == 0
        x_na = torch.full((p, n), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        rc = f(p, n, Rd.data_ptr(), Rd.stride(1), Rd.stride(0), yd.data_ptr(), yd.stride(0),
               x_na.data_ptr(), x_na.stride(0), tile, st.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert rc == 0, mdls.status_string(rc)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        got, ref = to_host(x_na), to_host(x_ws)
        assert np.all(np.isfinite(got))
        import oracle
        assert oracle.rel_err(got, ref) < TOL[p]


def test_noalloc_singular_status_and_oracle():
    """A zero on R's diagonal reaches the caller's status word; a regular
    problem matches the oracle's row-by-row back substitution."""
    import torch
    import oracle
    mdls, f = _entry()
    stream = torch.cuda.current_stream()
    p, n, tile = 2, 90, 32
    R, y = synth.upper_triangular(p, n, seed=23)
    for singular in (True, False):
        Rs = R.copy()
        if singular:
            Rs[:, 40, 40] = 0.0
        Rd, yd = to_dev(Rs), to_dev(y)
        x = torch.zeros((p, n), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        rc = f(p, n, Rd.data_ptr(), Rd.stride(1), Rd.stride(0), yd.data_ptr(), yd.stride(0),
               x.data_ptr(), x.stride(0), tile, st.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        if singular:
            assert int(st.item()) == mdls.MDLS_ERR_SINGULAR
        else:
            assert int(st.item()) == 0
            assert oracle.rel_err(to_host(x), oracle.backsub(R, y)) < TOL[p]


def test_noalloc_size_limits_quoted_in_the_header():
    """The largest n per precision at tile 128 that the header quotes fits
    the fixed scratch, and the next size up does not."""
    mdls, _ = _entry()
    limit = 16 << 20
    for p, n in ((2, 4960), (4, 2432), (8, 1152)):
        assert mdls.mdls_backsub_workspace(p, n, 128) <= limit
        assert mdls.mdls_backsub_workspace(p, n + 32, 128) > limit


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    mdls, f = _entry()
    limit = 16 << 20
    p, n = 8, 4096            # needs about 32 MiB of inverted tiles at tile 128
    assert mdls.mdls_backsub_workspace(p, n, 128) > limit
    R = torch.zeros((p, 1, 1), dtype=torch.float64, device="cuda")   # never read
    rc = f(p, n, R.data_ptr(), n, n * n, R.data_ptr(), n, R.data_ptr(), n, 128, None, None)
    assert rc == mdls.MDLS_ERR_WORKSPACE
