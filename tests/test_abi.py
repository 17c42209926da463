"""The C ABI library loads without a GPU and exports every entry point that
include/*.h declares; host-side argument checks return their codes before
any device work (no compute call is made here)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2110_08375_gb300 import build as b
    b.build()
    import paper_2110_08375_gb300 as pkg
    return pkg.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mdls_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mdls_qr", "mdls_backsub", "mdls_lstsq", "mdls_qr_workspace",
                     "mdls_backsub_workspace", "mdls_lstsq_workspace", "mdls_read_status",
                     "mdls_status_string", "mdls_vec_op", "mdls_version"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_and_status_strings(L):
    assert L.mdls_version() >= 100
    import paper_2110_08375_gb300 as pkg
    for code in range(-8, 1):
        s = pkg.status_string(code)
        assert s and s != "unknown status"
    assert pkg.status_string(-99) == "unknown status"


def test_workspace_queries(L):
    import paper_2110_08375_gb300 as pkg
    for p in (2, 4, 8):
        a = pkg.mdls_qr_workspace(p, 64, 48, 16, True)
        b = pkg.mdls_qr_workspace(p, 64, 48, 16, False)
        assert a > b > 0 and a % 256 == 0
        assert pkg.mdls_lstsq_workspace(p, 64, 48, 16) > 0
        assert pkg.mdls_backsub_workspace(p, 48, 16) > 0
    # more limbs need more space; invalid requests report 0
    assert pkg.mdls_qr_workspace(8, 64, 48, 16, True) > pkg.mdls_qr_workspace(2, 64, 48, 16, True)
    assert pkg.mdls_qr_workspace(3, 64, 48, 16, True) == 0
    assert pkg.mdls_qr_workspace(2, 40, 48, 16, True) == 0        # m < n
    assert pkg.mdls_qr_workspace(2, 64, 48, 300, True) == 0       # tile > 256
    assert pkg.mdls_qr_workspace(2, 64, 48, 16, True, mode=9) == 0
    assert pkg.mdls_backsub_workspace(2, 0, 16) == 0


def test_argument_errors_return_before_device_work(L):
    vp = C.c_void_p
    fake = vp(1 << 20)   # never dereferenced: every call below fails its host checks
    ws_bytes = 1 << 30
    # precision
    assert L.mdls_qr(3, 8, 4, fake, 8, 32, None, 0, 0, 2, 0, fake, ws_bytes, None) == -2
    # m < n, lda < m, plane stride too small, tile too large, bad mode
    assert L.mdls_qr(2, 4, 8, fake, 8, 64, None, 0, 0, 2, 0, fake, ws_bytes, None) == -1
    assert L.mdls_qr(2, 8, 4, fake, 4, 32, None, 0, 0, 2, 0, fake, ws_bytes, None) == -1
    assert L.mdls_qr(2, 8, 4, fake, 8, 16, None, 0, 0, 2, 0, fake, ws_bytes, None) == -1
    assert L.mdls_qr(2, 8, 4, fake, 8, 32, None, 0, 0, 999, 0, fake, ws_bytes, None) == -1
    assert L.mdls_qr(2, 8, 4, fake, 8, 32, None, 0, 0, 2, 7, fake, ws_bytes, None) == -1
    # workspace: NULL, too small, misaligned
    assert L.mdls_qr(2, 8, 4, fake, 8, 32, None, 0, 0, 2, 0, None, ws_bytes, None) == -3
    assert L.mdls_qr(2, 8, 4, fake, 8, 32, None, 0, 0, 2, 0, fake, 16, None) == -3
    assert L.mdls_qr(2, 8, 4, fake, 8, 32, None, 0, 0, 2, 0, vp((1 << 20) + 8), ws_bytes, None) == -3
    # back substitution and least squares
    assert L.mdls_backsub(5, 8, fake, 8, 64, fake, 8, fake, 8, 4, fake, ws_bytes, None) == -2
    assert L.mdls_backsub(2, 8, fake, 4, 64, fake, 8, fake, 8, 4, fake, ws_bytes, None) == -1
    assert L.mdls_backsub(2, 8, None, 8, 64, fake, 8, fake, 8, 4, fake, ws_bytes, None) == -1
    assert L.mdls_backsub(2, 8, fake, 8, 64, fake, 8, fake, 8, 4, fake, 8, None) == -3
    assert L.mdls_lstsq(2, 4, 8, fake, 8, 64, fake, 8, fake, 8, 4, 0, fake, ws_bytes, None) == -1
    assert L.mdls_lstsq(2, 8, 4, fake, 8, 32, fake, 4, fake, 4, 4, 0, fake, ws_bytes, None) == -1
    assert L.mdls_lstsq(2, 8, 4, fake, 8, 32, fake, 8, fake, 4, 4, 0, None, ws_bytes, None) == -3
    assert L.mdls_vec_op(2, 9, 4, fake, 4, fake, 4, fake, 4, None) == -1
    assert L.mdls_vec_op(6, 0, 4, fake, 4, fake, 4, fake, 4, None) == -2


def test_library_has_no_oracle_dependency():
    """The product library neither links nor names the oracle."""
    import subprocess
    from paper_2110_08375_gb300 import build as b
    lib = b.build()
    out = subprocess.run(["nm", "-D", lib], capture_output=True, text=True).stdout
    assert "mdref" not in out
    for src in glob.glob(os.path.join(ROOT, "paper_2110_08375_gb300", "**", "*"), recursive=True):
        if src.endswith((".cu", ".cuh", ".h", ".py")):
            text = open(src).read()
            assert "mdref" not in text and "import oracle" not in text, src


def test_wait_check_argument_errors(L):
    vp = C.c_void_p
    fake = vp(1 << 20)
    L.mdls_wait_check.argtypes = [vp, C.c_size_t, C.c_uint64, C.c_int, vp]
    assert L.mdls_wait_check(None, 512, 10**6, 0, None) == -3
    assert L.mdls_wait_check(fake, 256, 10**6, 0, None) == -3          # too small
    assert L.mdls_wait_check(vp((1 << 20) + 64), 512, 10**6, 0, None) == -3   # misaligned
    assert L.mdls_wait_check(fake, 512, 10, 0, None) == -1             # limit below 1 us
    assert L.mdls_wait_check(fake, 512, 2 * 10**10, 0, None) == -1     # limit above 10 s
    assert L.mdls_wait_check(fake, 512, 10**6, 2, None) == -1


def test_backsub_schedule_argument(L):
    import paper_2110_08375_gb300 as pkg
    assert L.mdls_set_backsub_schedule(3) == -1
    assert L.mdls_set_backsub_schedule(-1) == -1
    for s in (pkg.BS_PER_STEP, pkg.BS_PERSISTENT, pkg.BS_AUTO):
        assert L.mdls_set_backsub_schedule(s) == 0


def test_split_engine_argument(L):
    import paper_2110_08375_gb300 as pkg
    assert L.mdls_set_split_engine(3) == -1
    assert L.mdls_set_split_engine(-1) == -1
    for e in (pkg.SPLIT_ENGINE_MMA_SYNC, pkg.SPLIT_ENGINE_TCGEN05, pkg.SPLIT_ENGINE_AUTO):
        assert L.mdls_set_split_engine(e) == 0


def test_toeplitz_argument_errors(L):
    vp = C.c_void_p
    fake = vp(1 << 20)
    ws_bytes = 1 << 30
    # m < n, negative d, block stride too small, precision
    assert L.mdls_toeplitz_lstsq(2, 4, 8, 1, fake, 4, 64, 32, fake, 8, 4, fake, 16, 8, 4, fake, ws_bytes, None) == -1
    assert L.mdls_toeplitz_lstsq(2, 8, 4, -1, fake, 8, 64, 32, fake, 16, 8, fake, 8, 4, 4, fake, ws_bytes, None) == -1
    assert L.mdls_toeplitz_lstsq(2, 8, 4, 1, fake, 8, 64, 16, fake, 16, 8, fake, 8, 4, 4, fake, ws_bytes, None) == -1
    assert L.mdls_toeplitz_lstsq(3, 8, 4, 1, fake, 8, 64, 32, fake, 16, 8, fake, 8, 4, 4, fake, ws_bytes, None) == -2
    assert L.mdls_toeplitz_lstsq(2, 8, 4, 1, fake, 8, 64, 32, fake, 16, 8, fake, 8, 4, 4, None, ws_bytes, None) == -3
