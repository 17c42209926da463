"""Multiple-double least squares on one GB300 (arXiv 2110.08375), CUDA path.

This module is a thin ctypes binding of ``libmdls.so`` (C ABI declared in
``include/mdls.h``): it marshals torch tensors to device pointers, sizes and
strides, and raises on error codes.  Every step of the computation runs in the
library's CUDA kernels; there is no CPU fallback.  If the library is missing
or no GPU is present, calls fail loudly.

Tensor convention (limb-planar, as in the paper's Section 2): an md matrix
with ``rows x cols`` entries is a float64 CUDA tensor of shape
``(p, cols, ld)`` whose planes are column-major (``ld >= rows``); a vector of
length n is ``(p, n)``.  p = 2 (double double), 4 (quad double), 8 (octo
double).
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmdls.so")

MDLS_OK = 0
MDLS_ERR_ARG = -1
MDLS_ERR_PREC = -2
MDLS_ERR_WORKSPACE = -3
MDLS_ERR_SINGULAR = -4
MDLS_ERR_CUDA = -5
MDLS_ERR_TIMEOUT = -6
MDLS_ERR_UNSUPPORTED = -7
MDLS_ERR_NOT_CONVERGED = -8
MODE_PLAIN = 0
MODE_SPLIT = 1
MODE_REFINE = 2
OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "fma": 4, "sqrt": 5}

_lib = None


class Problem(C.Structure):
    """mdls_problem of include/mdls.h."""
    _fields_ = [("prec", C.c_int), ("tile", C.c_int), ("m", C.c_int64), ("n", C.c_int64),
                ("A", C.c_void_p), ("lda", C.c_int64), ("psa", C.c_int64),
                ("b", C.c_void_p), ("psb", C.c_int64), ("x", C.c_void_p), ("psx", C.c_int64)]


class MdlsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


def lib() -> C.CDLL:
    """Loads libmdls.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmdls.so not built at {LIB_PATH}; run paper_2110_08375_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    i64, vp, sz = C.c_int64, C.c_void_p, C.c_size_t
    L.mdls_version.restype = C.c_int
    L.mdls_status_string.restype = C.c_char_p
    L.mdls_status_string.argtypes = [C.c_int]
    L.mdls_qr.argtypes = [C.c_int, i64, i64, vp, i64, i64, vp, i64, i64, C.c_int, C.c_int, vp, sz, vp]
    L.mdls_qr_workspace.argtypes = [C.c_int, i64, i64, C.c_int, C.c_int, C.c_int]
    L.mdls_qr_workspace.restype = sz
    L.mdls_backsub.argtypes = [C.c_int, i64, vp, i64, i64, vp, i64, vp, i64, C.c_int, vp, sz, vp]
    L.mdls_backsub_workspace.argtypes = [C.c_int, i64, C.c_int]
    L.mdls_backsub_workspace.restype = sz
    L.mdls_lstsq.argtypes = [C.c_int, i64, i64, vp, i64, i64, vp, i64, vp, i64, C.c_int, C.c_int, vp,
                             sz, vp]
    L.mdls_lstsq_workspace.argtypes = [C.c_int, i64, i64, C.c_int, C.c_int]
    L.mdls_lstsq_workspace.restype = sz
    L.mdls_read_status.argtypes = [vp, C.POINTER(C.c_int), vp]
    L.mdls_profile_enable.argtypes = [C.c_int]
    L.mdls_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]
    L.mdls_stage_name.argtypes = [C.c_int]
    L.mdls_stage_name.restype = C.c_char_p
    L.mdls_batched_workspace.argtypes = [C.POINTER(Problem), C.c_int]
    L.mdls_batched_workspace.restype = sz
    L.mdls_batched_plan.argtypes = [C.POINTER(Problem), C.c_int, vp, sz, C.c_int, C.POINTER(vp)]
    L.mdls_batched_launch.argtypes = [vp, vp]
    L.mdls_batched_status.argtypes = [vp, C.POINTER(C.c_int), vp]
    L.mdls_batched_tiles.argtypes = [vp, C.POINTER(C.c_int)]
    L.mdls_batched_modes.argtypes = [vp, C.POINTER(C.c_int)]
    L.mdls_batched_destroy.argtypes = [vp]
    L.mdls_batched_destroy.restype = None
    L.mdls_lstsq_batched_workspace.argtypes = [vp, C.c_int]
    L.mdls_lstsq_batched_workspace.restype = sz
    L.mdls_lstsq_batched.argtypes = [vp, C.c_int, vp, sz, vp, vp]
    L.mdls_vec_op.argtypes = [C.c_int, C.c_int, i64, vp, i64, vp, i64, vp, i64, vp]
    L.mdls_wait_check.argtypes = [vp, sz, C.c_uint64, C.c_int, vp]
    L.mdls_set_backsub_schedule.argtypes = [C.c_int]
    L.mdls_set_split_engine.argtypes = [C.c_int]
    L.mdls_toeplitz_lstsq_workspace.argtypes = [C.c_int, i64, i64, C.c_int]
    L.mdls_toeplitz_lstsq_workspace.restype = sz
    L.mdls_toeplitz_lstsq.argtypes = [C.c_int, i64, i64, i64, vp, i64, i64, i64, vp, i64, i64, vp, i64, i64,
                                      C.c_int, vp, sz, vp]
    L.mdls_zqr.argtypes = [C.c_int, i64, i64, vp, vp, i64, i64, vp, vp, i64, i64, C.c_int, vp, sz, vp]
    L.mdls_zqr_workspace.argtypes = [C.c_int, i64, i64, C.c_int, C.c_int]
    L.mdls_zqr_workspace.restype = sz
    L.mdls_zbacksub.argtypes = [C.c_int, i64, vp, vp, i64, i64, vp, vp, i64, vp, vp, i64, C.c_int, vp, sz, vp]
    L.mdls_zbacksub_workspace.argtypes = [C.c_int, i64, C.c_int]
    L.mdls_zbacksub_workspace.restype = sz
    L.mdls_zlstsq.argtypes = [C.c_int, i64, i64, vp, vp, i64, i64, vp, vp, i64, vp, vp, i64, C.c_int, vp, sz,
                              vp]
    L.mdls_zlstsq_workspace.argtypes = [C.c_int, i64, i64, C.c_int]
    L.mdls_zlstsq_workspace.restype = sz
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().mdls_status_string(int(code)).decode()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the multiple-double CUDA path needs a CUDA GPU")
    return torch


def _check_md(t, ndim: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if t.dim() != ndim or t.shape[0] not in (2, 4, 8):
        raise ValueError(f"{name} must have shape (p, ...) with p in (2, 4, 8) and {ndim} dims")
    if t.stride(-1) != 1:
        raise ValueError(f"{name}: innermost dimension must be contiguous")


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def workspace(nbytes: int, device=None):
    """A 256-byte aligned device buffer of at least nbytes (torch allocation)."""
    torch = _torch()
    buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-buf.data_ptr()) % 256
    return buf[off:off + int(nbytes)]


def mdls_qr_workspace(prec: int, m: int, n: int, tile: int = 0, want_q: bool = True,
                      mode: int = MODE_PLAIN) -> int:
    return int(lib().mdls_qr_workspace(prec, m, n, tile, int(want_q), mode))


def mdls_backsub_workspace(prec: int, n: int, tile: int = 0) -> int:
    return int(lib().mdls_backsub_workspace(prec, n, tile))


def mdls_lstsq_workspace(prec: int, m: int, n: int, tile: int = 0, mode: int = MODE_PLAIN) -> int:
    return int(lib().mdls_lstsq_workspace(prec, m, n, tile, mode))


def mdls_qr(A, Q=None, rows: int | None = None, tile: int = 0, mode: int = MODE_PLAIN, ws=None,
            stream=None):
    """In-place blocked Householder QR (Algorithm 2).  A: (p, n, ld); on return
    its upper triangle is R and the rest zero.  Q: (p, m, ldq) or None."""
    _check_md(A, 3, "A")
    p, n, lda = A.shape
    m = lda if rows is None else int(rows)
    if Q is not None:
        _check_md(Q, 3, "Q")
    need = mdls_qr_workspace(p, m, n, tile, Q is not None, mode)
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_qr_workspace")
    if ws is None:
        ws = workspace(need, A.device)
    rc = lib().mdls_qr(p, m, n, A.data_ptr(), A.stride(1), A.stride(0),
                       Q.data_ptr() if Q is not None else None,
                       Q.stride(1) if Q is not None else 0, Q.stride(0) if Q is not None else 0,
                       tile, mode, ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_qr")
    return ws


def mdls_backsub(R, y, x, tile: int = 0, ws=None, stream=None):
    """Algorithm 1: solves R x = y (R: (p, n, ld) upper triangular; y, x: (p, n))."""
    _check_md(R, 3, "R"); _check_md(y, 2, "y"); _check_md(x, 2, "x")
    p, n, ldr = R.shape
    need = mdls_backsub_workspace(p, n, tile)
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_backsub_workspace")
    if ws is None:
        ws = workspace(need, R.device)
    rc = lib().mdls_backsub(p, n, R.data_ptr(), R.stride(1), R.stride(0), y.data_ptr(), y.stride(0),
                            x.data_ptr(), x.stride(0), tile, ws.data_ptr(),
                            ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_backsub")
    return ws


def mdls_lstsq(A, b, x, rows: int | None = None, tile: int = 0, mode: int = MODE_PLAIN, ws=None,
               stream=None):
    """Least squares min ||b - A x|| (A: (p, n, ld), b: (p, m), x: (p, n))."""
    _check_md(A, 3, "A"); _check_md(b, 2, "b"); _check_md(x, 2, "x")
    p, n, lda = A.shape
    m = lda if rows is None else int(rows)
    need = mdls_lstsq_workspace(p, m, n, tile, mode)
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_lstsq_workspace")
    if ws is None:
        ws = workspace(need, A.device)
    rc = lib().mdls_lstsq(p, m, n, A.data_ptr(), A.stride(1), A.stride(0), b.data_ptr(), b.stride(0),
                          x.data_ptr(), x.stride(0), tile, mode, ws.data_ptr(),
                          ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_lstsq")
    return ws


def mdls_toeplitz_lstsq(J, b, x, rows: int | None = None, tile: int = 0, ws=None, stream=None):
    """Block-Toeplitz power-series solve: J (p, d+1, n, ld) blocks J_0..J_d,
    b (p, d+1, m), x (p, d+1, n) receives x_0..x_d of J(t) x(t) = b(t) mod
    t^{d+1} (least squares per block with one QR of J_0)."""
    import torch
    for t, nm in ((J, "J"), (b, "b"), (x, "x")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.stride(-1) != 1:
            raise TypeError(f"{nm} must be a float64 CUDA tensor with contiguous rows")
    if J.dim() != 4 or b.dim() != 3 or x.dim() != 3:
        raise ValueError("J must be (p, d+1, n, ld), b (p, d+1, m), x (p, d+1, n)")
    p, d1, n, ldj = J.shape
    m = ldj if rows is None else int(rows)
    need = int(lib().mdls_toeplitz_lstsq_workspace(p, m, n, tile))
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_toeplitz_lstsq_workspace")
    if ws is None:
        ws = workspace(need, J.device)
    rc = lib().mdls_toeplitz_lstsq(p, m, n, d1 - 1, J.data_ptr(), J.stride(2), J.stride(0), J.stride(1),
                                   b.data_ptr(), b.stride(0), b.stride(1), x.data_ptr(), x.stride(0), x.stride(1),
                                   tile, ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_toeplitz_lstsq")
    return ws


def _same_layout(a, b, name):
    if a.shape != b.shape or a.stride() != b.stride():
        raise ValueError(f"{name}: real and imaginary parts must have one shape and one layout")


def mdls_zqr(Ar, Ai, Qr=None, Qi=None, rows: int | None = None, tile: int = 0, ws=None, stream=None):
    """In-place complex blocked Householder QR: (Ar, Ai) (p, n, ld) become R
    (strictly lower part zero); (Qr, Qi) (p, m, ldq) receive Q, or None."""
    _check_md(Ar, 3, "Ar"); _check_md(Ai, 3, "Ai"); _same_layout(Ar, Ai, "A")
    p, n, lda = Ar.shape
    m = lda if rows is None else int(rows)
    want_q = Qr is not None
    if want_q:
        _check_md(Qr, 3, "Qr"); _check_md(Qi, 3, "Qi"); _same_layout(Qr, Qi, "Q")
    need = int(lib().mdls_zqr_workspace(p, m, n, tile, int(want_q)))
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_zqr_workspace")
    if ws is None:
        ws = workspace(need, Ar.device)
    rc = lib().mdls_zqr(p, m, n, Ar.data_ptr(), Ai.data_ptr(), Ar.stride(1), Ar.stride(0),
                        Qr.data_ptr() if want_q else None, Qi.data_ptr() if want_q else None,
                        Qr.stride(1) if want_q else 0, Qr.stride(0) if want_q else 0, tile, ws.data_ptr(),
                        ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_zqr")
    return ws


def mdls_zbacksub(Rr, Ri, yr, yi, xr, xi, tile: int = 0, ws=None, stream=None):
    """Algorithm 1 on complex data: solves R x = y (R: (p, n, ld) parts; y, x: (p, n) parts)."""
    for t, nd, nm in ((Rr, 3, "Rr"), (Ri, 3, "Ri"), (yr, 2, "yr"), (yi, 2, "yi"), (xr, 2, "xr"), (xi, 2, "xi")):
        _check_md(t, nd, nm)
    _same_layout(Rr, Ri, "R"); _same_layout(yr, yi, "y"); _same_layout(xr, xi, "x")
    p, n, ldr = Rr.shape
    need = int(lib().mdls_zbacksub_workspace(p, n, tile))
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_zbacksub_workspace")
    if ws is None:
        ws = workspace(need, Rr.device)
    rc = lib().mdls_zbacksub(p, n, Rr.data_ptr(), Ri.data_ptr(), Rr.stride(1), Rr.stride(0), yr.data_ptr(),
                             yi.data_ptr(), yr.stride(0), xr.data_ptr(), xi.data_ptr(), xr.stride(0), tile,
                             ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_zbacksub")
    return ws


def mdls_zlstsq(Ar, Ai, br, bi, xr, xi, rows: int | None = None, tile: int = 0, ws=None, stream=None):
    """Complex least squares min ||b - A x|| (A: (p, n, ld) parts; b (p, m), x (p, n) parts)."""
    for t, nd, nm in ((Ar, 3, "Ar"), (Ai, 3, "Ai"), (br, 2, "br"), (bi, 2, "bi"), (xr, 2, "xr"), (xi, 2, "xi")):
        _check_md(t, nd, nm)
    _same_layout(Ar, Ai, "A"); _same_layout(br, bi, "b"); _same_layout(xr, xi, "x")
    p, n, lda = Ar.shape
    m = lda if rows is None else int(rows)
    need = int(lib().mdls_zlstsq_workspace(p, m, n, tile))
    if need == 0:
        raise MdlsError(MDLS_ERR_ARG, "mdls_zlstsq_workspace")
    if ws is None:
        ws = workspace(need, Ar.device)
    rc = lib().mdls_zlstsq(p, m, n, Ar.data_ptr(), Ai.data_ptr(), Ar.stride(1), Ar.stride(0), br.data_ptr(),
                           bi.data_ptr(), br.stride(0), xr.data_ptr(), xi.data_ptr(), xr.stride(0), tile,
                           ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_zlstsq")
    return ws


def mdls_read_status(ws, stream=None) -> int:
    """Synchronises the stream and returns the device status word of ws."""
    st = C.c_int(0)
    rc = lib().mdls_read_status(ws.data_ptr(), C.byref(st), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_read_status")
    return st.value


def mdls_vec_op(op: str, a, b=None, c=None, stream=None):
    """Elementwise md arithmetic: c = a op b (op in add, sub, mul, div, fma:
    c = c + a*b, sqrt: c = sqrt(a)).  a, b, c: (p, n) tensors."""
    torch = _torch()
    _check_md(a, 2, "a")
    if c is None:
        c = torch.zeros_like(a)
    bb = a if b is None else b
    rc = lib().mdls_vec_op(a.shape[0], OPS[op], a.shape[1], a.data_ptr(), a.stride(0),
                           bb.data_ptr(), bb.stride(0), c.data_ptr(), c.stride(0), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_vec_op")
    return c


BS_AUTO, BS_PER_STEP, BS_PERSISTENT = 0, 1, 2


def mdls_set_backsub_schedule(schedule: int) -> None:
    """Step 2 of the back substitution per tile step (BS_PER_STEP), in one
    persistent launch (BS_PERSISTENT) or chosen by size (BS_AUTO)."""
    rc = lib().mdls_set_backsub_schedule(int(schedule))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_set_backsub_schedule")


WAIT_CHECK_WORKSPACE = 512


SPLIT_ENGINE_AUTO, SPLIT_ENGINE_MMA_SYNC, SPLIT_ENGINE_TCGEN05 = 0, 1, 2


def mdls_set_split_engine(engine: int) -> None:
    """Kernel of the split-mode digit products: tcgen05 (SPLIT_ENGINE_TCGEN05),
    mma.sync (SPLIT_ENGINE_MMA_SYNC) or chosen by shape (SPLIT_ENGINE_AUTO)."""
    rc = lib().mdls_set_split_engine(int(engine))
    if rc != 0:
        raise MdlsError(rc, "mdls_set_split_engine")


def mdls_wait_check(limit_ns: int, publish: bool, ws=None, stream=None):
    """Runs the library's bounded device wait with the given limit on a flag
    that is published (publish=True) or never published; returns the
    workspace, whose status then reads MDLS_OK or MDLS_ERR_TIMEOUT."""
    if ws is None:
        ws = workspace(WAIT_CHECK_WORKSPACE)
    rc = lib().mdls_wait_check(ws.data_ptr(), ws.numel() * ws.element_size(), int(limit_ns),
                               int(bool(publish)), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_wait_check")
    return ws


N_STAGES = 9
STAGE_KEYS = ("panel", "compute_w", "trailing", "q_accum", "invert_tiles", "mul_inverses",
              "bs_update", "other", "refine")


def mdls_profile_enable(on: bool = True) -> None:
    lib().mdls_profile_enable(int(bool(on)))


def mdls_profile_read() -> dict:
    """Per-stage (milliseconds, launches) since the last read; resets them."""
    ms = (C.c_double * N_STAGES)()
    cnt = (C.c_int64 * N_STAGES)()
    rc = lib().mdls_profile_read(ms, cnt, N_STAGES)
    if rc < 0:
        raise MdlsError(rc, "mdls_profile_read")
    return {k: (ms[i], int(cnt[i])) for i, k in enumerate(STAGE_KEYS)}


def mdls_stage_name(stage: int) -> str:
    return lib().mdls_stage_name(int(stage)).decode()



class BatchedPlan:
    """A plan of mdls_batched_plan: one graph launch solves every problem.

    problems: list of (A, b, x) or (A, b, x, tile) tensors, A (p, n, ld),
    b (p, m), x (p, n) on the GPU.  The plan keeps references to them and to
    its workspace, which must not be freed while the plan lives.
    """

    def __init__(self, problems, autotune: bool = True):
        torch = _torch()
        arr = (Problem * len(problems))()
        self._keep = []
        for i, pr in enumerate(problems):
            A, b, x = pr[:3]
            tile = pr[3] if len(pr) > 3 else 0
            for t, nd, nm in ((A, 3, "A"), (b, 2, "b"), (x, 2, "x")):
                _check_md(t, nd, nm)
            p, n, lda = A.shape
            arr[i] = Problem(p, tile, lda, n, A.data_ptr(), A.stride(1), A.stride(0), b.data_ptr(),
                             b.stride(0), x.data_ptr(), x.stride(0))
            self._keep.append((A, b, x))
        self.count = len(problems)
        need = lib().mdls_batched_workspace(arr, self.count)
        if need == 0:
            raise MdlsError(MDLS_ERR_ARG, "mdls_batched_workspace")
        self.ws = workspace(need, self._keep[0][0].device)
        handle = C.c_void_p()
        torch.cuda.synchronize()
        rc = lib().mdls_batched_plan(arr, self.count, self.ws.data_ptr(), need, int(autotune), C.byref(handle))
        if rc != MDLS_OK:
            raise MdlsError(rc, "mdls_batched_plan")
        self.handle = handle
        self._arr = arr

    def launch(self, stream=None):
        rc = lib().mdls_batched_launch(self.handle, _stream(stream))
        if rc != MDLS_OK:
            raise MdlsError(rc, "mdls_batched_launch")

    def status(self, stream=None):
        out = (C.c_int * self.count)()
        rc = lib().mdls_batched_status(self.handle, out, _stream(stream))
        if rc != MDLS_OK:
            raise MdlsError(rc, "mdls_batched_status")
        return list(out)

    def tiles(self):
        out = (C.c_int * self.count)()
        lib().mdls_batched_tiles(self.handle, out)
        return list(out)

    def modes(self):
        out = (C.c_int * self.count)()
        lib().mdls_batched_modes(self.handle, out)
        return list(out)

    def destroy(self):
        if getattr(self, "handle", None):
            lib().mdls_batched_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def mdls_batched_plan(problems, autotune: bool = True) -> BatchedPlan:
    return BatchedPlan(problems, autotune)


def problems_device(problems, device=None):
    """The mdls_problem records of problems [(A, b, x) or (A, b, x, tile)]
    as a device byte tensor (the layout of include/mdls.h)."""
    torch = _torch()
    arr = (Problem * len(problems))()
    for i, pr in enumerate(problems):
        A, b, x = pr[:3]
        tile = pr[3] if len(pr) > 3 else 0
        for t, nd, nm in ((A, 3, "A"), (b, 2, "b"), (x, 2, "x")):
            _check_md(t, nd, nm)
        p, n, lda = A.shape
        arr[i] = Problem(p, tile, lda, n, A.data_ptr(), A.stride(1), A.stride(0), b.data_ptr(), b.stride(0),
                         x.data_ptr(), x.stride(0))
    raw = bytes(memoryview(arr).cast("B"))
    host = torch.frombuffer(bytearray(raw), dtype=torch.uint8)
    return host.to(device or problems[0][0].device)


def mdls_lstsq_batched(problems, ws=None, status=None, probs_dev=None, stream=None):
    """Solves every problem with one call (mdls_lstsq_batched): the problem
    array and the per-problem status live on the device.  Returns
    (ws, status) -- keep ws (and the problems' tensors) for repeated calls:
    the library caches the plan of a batch by its contents and workspace."""
    torch = _torch()
    if probs_dev is None:
        probs_dev = problems_device(problems)
    count = len(problems)
    if ws is None:
        need = lib().mdls_lstsq_batched_workspace(probs_dev.data_ptr(), count)
        if need == 0:
            raise MdlsError(MDLS_ERR_ARG, "mdls_lstsq_batched_workspace")
        ws = workspace(need, probs_dev.device)
    if status is None:
        status = torch.full((count,), -99, dtype=torch.int32, device=probs_dev.device)
    rc = lib().mdls_lstsq_batched(probs_dev.data_ptr(), count, ws.data_ptr(), ws.numel() * ws.element_size(),
                                  status.data_ptr(), _stream(stream))
    if rc != MDLS_OK:
        raise MdlsError(rc, "mdls_lstsq_batched")
    return ws, status

