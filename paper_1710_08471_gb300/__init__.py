"""GB300-native CholeskyQR2 (Hutter & Solomonik, arXiv 1710.08471).

Thin Python binding of the C ABI in include/cqr2.h. Every function here only
marshals arguments (device pointers, leading dimensions, the current CUDA
stream) into libcqr2.so, whose CUDA kernels do all the arithmetic. PyTorch is
used for device memory and streams only.

Matrices are column-major like the C ABI: an m x n matrix is a torch tensor of
shape (m, n) with stride (1, ld), ld >= m. ``colmajor`` and ``empty_colmajor``
make such tensors.
"""
from __future__ import annotations

import ctypes as C

from . import _native as N
from ._native import (  # noqa: F401
    CQR2_ERR_CUDA,
    CQR2_ERR_INVALID_ARG,
    CQR2_ERR_NOT_SPD,
    CQR2_ERR_OOM,
    CQR2_ERR_TIMEOUT,
    CQR2_ERR_UNSUPPORTED,
    CQR2_FP64,
    CQR2_FUSED,
    CQR2_OK,
    CQR2_OZAKI_BF16,
    CQR2_OZAKI_BF16_S6,
    CQR2Error,
    Info,
)

__all__ = [
    "Plan", "colmajor", "empty_colmajor", "factor", "lstsq", "cqr2_plan_create", "cqr2_factor", "cqr2_lstsq",
    "cqr2_syrk", "cqr2_cholinv", "cqr2_qform", "cqr2_trmm_upper", "cqr2_workspace_bytes", "cqr2_plan_destroy",
    "cqr2_plan_info", "library_path", "cqr2_factor_host", "cqr2_plan_set_profiling", "cqr2_plan_stage_times",
    "cqr2_launch_count",
]


def library_path() -> str:
    return N.LIB_PATH


def _torch():
    import torch
    return torch


def empty_colmajor(m: int, n: int, device=None, dtype=None):
    """Uninitialised m x n column-major tensor (stride (1, m))."""
    torch = _torch()
    return torch.empty((n, m), device=device, dtype=dtype or torch.float64).t()


def colmajor(x):
    """Column-major copy of a 2-D tensor (returned as-is if already so)."""
    if x.dim() == 2 and x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
        return x
    return x.t().contiguous().t()


def _mat(x, rows: int, cols: int, name: str):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if tuple(x.shape) != (rows, cols):
        raise ValueError(f"{name} must be {rows} x {cols}, got {tuple(x.shape)}")
    if cols > 1 and x.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride (1, ld))")
    ld = x.stride(1) if cols > 1 else max(rows, 1)
    return C.c_void_p(x.data_ptr()), ld


def _vec(x, n: int, name: str):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if x.numel() != n or (n > 1 and x.stride(-1) != 1) or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous vector of length {n}")
    return C.c_void_p(x.data_ptr())


def _stream_handle(stream=None) -> C.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ----------------------------------------------------------- raw C ABI

def cqr2_plan_create(m: int, n: int, precision: int = CQR2_FP64, flags: int = 0, stream=None) -> C.c_void_p:
    lib = N.load()
    h = C.c_void_p()
    N.check(lib.cqr2_plan_create(C.byref(h), m, n, precision, flags, _stream_handle(stream)), "cqr2_plan_create")
    return h


def cqr2_plan_destroy(plan) -> None:
    N.load().cqr2_plan_destroy(plan)


def cqr2_workspace_bytes(plan) -> int:
    return int(N.load().cqr2_workspace_bytes(plan))


def cqr2_plan_info(plan) -> Info:
    info = Info()
    st = N.load().cqr2_plan_info(plan, C.byref(info))
    if st not in (CQR2_OK, CQR2_ERR_NOT_SPD):
        N.check(st, "cqr2_plan_info")
    return info


def cqr2_factor(plan, m, n, A, Q, R, sync: bool = True) -> Info | None:
    a, lda = _mat(A, m, n, "A")
    q, ldq = _mat(Q, m, n, "Q")
    r, ldr = _mat(R, n, n, "R")
    info = Info() if sync else None
    st = N.load().cqr2_factor(plan, a, lda, q, ldq, r, ldr, C.byref(info) if sync else None)
    N.check(st, "cqr2_factor", info)
    return info


def cqr2_lstsq(plan, m, n, A, b, x, Q, R=None, sync: bool = True) -> Info | None:
    a, lda = _mat(A, m, n, "A")
    q, ldq = _mat(Q, m, n, "Q")
    if R is not None:
        r, ldr = _mat(R, n, n, "R")
    else:
        r, ldr = None, n
    info = Info() if sync else None
    st = N.load().cqr2_lstsq(plan, a, lda, _vec(b, m, "b"), _vec(x, n, "x"), q, ldq, r, ldr,
                             C.byref(info) if sync else None)
    N.check(st, "cqr2_lstsq", info)
    return info


def cqr2_factor_rows(plan, m, n, A, Q, R, sync: bool = True) -> Info | None:
    """cqr2_factor for an m-row matrix on a plan created for at least m rows."""
    a, lda = _mat(A, m, n, "A")
    q, ldq = _mat(Q, m, n, "Q")
    r, ldr = _mat(R, n, n, "R")
    info = Info() if sync else None
    st = N.load().cqr2_factor_rows(plan, m, a, lda, q, ldq, r, ldr, C.byref(info) if sync else None)
    N.check(st, "cqr2_factor_rows", info)
    return info


def cqr2_lstsq_rows(plan, m, n, A, b, x, Q, R=None, sync: bool = True) -> Info | None:
    """cqr2_lstsq for an m-row matrix on a plan created for at least m rows."""
    a, lda = _mat(A, m, n, "A")
    if Q is not None:
        q, ldq = _mat(Q, m, n, "Q")
    else:
        q, ldq = None, m  # Q into the plan's own buffer
    if R is not None:
        r, ldr = _mat(R, n, n, "R")
    else:
        r, ldr = None, n
    info = Info() if sync else None
    st = N.load().cqr2_lstsq_rows(plan, m, a, lda, _vec(b, m, "b"), _vec(x, n, "x"), q, ldq, r, ldr,
                                  C.byref(info) if sync else None)
    N.check(st, "cqr2_lstsq_rows", info)
    return info


def cqr2_syrk(plan, m, n, A, W) -> None:
    a, lda = _mat(A, m, n, "A")
    w, ldw = _mat(W, n, n, "W")
    N.check(N.load().cqr2_syrk(plan, a, lda, w, ldw), "cqr2_syrk")


def cqr2_cholinv(plan, n, W, L, Y, sync: bool = True) -> Info | None:
    w, ldw = _mat(W, n, n, "W")
    l_, ldl = _mat(L, n, n, "L")
    y, ldy = _mat(Y, n, n, "Y")
    info = Info() if sync else None
    st = N.load().cqr2_cholinv(plan, w, ldw, l_, ldl, y, ldy, C.byref(info) if sync else None)
    N.check(st, "cqr2_cholinv", info)
    return info


def cqr2_qform(plan, m, n, A, Rinv, Q) -> None:
    a, lda = _mat(A, m, n, "A")
    ri, ldri = _mat(Rinv, n, n, "Rinv")
    q, ldq = _mat(Q, m, n, "Q")
    N.check(N.load().cqr2_qform(plan, a, lda, ri, ldri, q, ldq), "cqr2_qform")


def cqr2_trmm_upper(plan, n, R2, R1, R) -> None:
    r2, ld2 = _mat(R2, n, n, "R2")
    r1, ld1 = _mat(R1, n, n, "R1")
    r, ldr = _mat(R, n, n, "R")
    N.check(N.load().cqr2_trmm_upper(plan, r2, ld2, r1, ld1, r, ldr), "cqr2_trmm_upper")


def cqr2_syrk_noalloc(m, n, A, W, stream=None) -> None:
    """W = A^T A without any device allocation (fixed library scratch); for
    callers that must not allocate device memory. n <= 2816."""
    a, lda = _mat(A, m, n, "A")
    w, ldw = _mat(W, n, n, "W")
    N.check(N.load().cqr2_syrk_noalloc(a, m, n, lda, w, ldw, _stream_handle(stream)), "cqr2_syrk_noalloc")


def cqr2_factor_host(plan, m, n, hA, hQ, hR) -> Info:
    """Host-buffer CholeskyQR2. hA, hQ, hR are Fortran-ordered float64 numpy
    arrays (pinned or pageable) of shapes (m, n), (m, n), (n, n)."""
    import numpy as np

    for name, x, shape in (("A", hA, (m, n)), ("Q", hQ, (m, n)), ("R", hR, (n, n))):
        if not isinstance(x, np.ndarray) or x.dtype != np.float64 or x.shape != shape:
            raise TypeError(f"{name} must be a float64 numpy array of shape {shape}")
        if not x.flags.f_contiguous:
            raise ValueError(f"{name} must be column-major (Fortran order)")
    info = Info()
    st = N.load().cqr2_factor_host(plan, hA.ctypes.data, m, hQ.ctypes.data, m, hR.ctypes.data, n, C.byref(info))
    N.check(st, "cqr2_factor_host", info)
    return info


def cqr2_plan_set_profiling(plan, enable: bool) -> None:
    N.check(N.load().cqr2_plan_set_profiling(plan, 1 if enable else 0), "cqr2_plan_set_profiling")


def cqr2_plan_stage_times(plan) -> dict:
    """{stage name: (total ms, count)} since profiling was enabled."""
    lib = N.load()
    ms = (C.c_double * N.CQR2_NUM_STAGES)()
    cnt = (C.c_int64 * N.CQR2_NUM_STAGES)()
    N.check(lib.cqr2_plan_stage_times(plan, ms, cnt, N.CQR2_NUM_STAGES), "cqr2_plan_stage_times")
    return {lib.cqr2_stage_name(i).decode(): (ms[i], int(cnt[i])) for i in range(N.CQR2_NUM_STAGES)}


def cqr2_launch_count() -> int:
    return int(N.load().cqr2_launch_count())


def cqr2_plan_set_gram_ctas(plan, ctas_per_sm: int) -> None:
    N.check(N.load().cqr2_plan_set_gram_ctas(plan, ctas_per_sm), "cqr2_plan_set_gram_ctas")


def cqr2_plan_set_fused(plan, fused: bool) -> None:
    N.check(N.load().cqr2_plan_set_fused(plan, 1 if fused else 0), "cqr2_plan_set_fused")


def cqr2_plan_set_inverse_depth(plan, depth: int) -> None:
    """Triangular inverse only on the diagonal blocks below the top `depth`
    halvings of CholInv; L21 and Q by block forward substitution."""
    N.check(N.load().cqr2_plan_set_inverse_depth(plan, int(depth)), "cqr2_plan_set_inverse_depth")


def cqr2_autotune(m: int, n: int, precision: int = CQR2_FP64) -> dict:
    """Time candidate plan configurations for an m x n factorization and
    record the best in the library's tuning table."""
    res = N.TuneResult()
    N.check(N.load().cqr2_autotune(m, n, precision, C.byref(res)), "cqr2_autotune")
    return {"gram_ctas": res.gram_ctas, "fused": bool(res.fused), "ms": res.ms, "candidates": res.candidates}


def cqr2_autotune_batch(n: int, count: int) -> int:
    """Time a batch of `count` problems of width n through the grouped kernel
    and through plans for doubling m, and set the routing limit on m n^2 used
    by batches created later; returns it."""
    lim = C.c_int64()
    N.check(N.load().cqr2_autotune_batch(int(n), int(count), C.byref(lim)), "cqr2_autotune_batch")
    return lim.value


def cqr2_tune_set_small_limit(limit: int) -> None:
    N.check(N.load().cqr2_tune_set_small_limit(int(limit)), "cqr2_tune_set_small_limit")


def cqr2_tune_table() -> str:
    lib = N.load()
    size = int(lib.cqr2_tune_table(None, 0))
    buf = C.create_string_buffer(size)
    lib.cqr2_tune_table(buf, size)
    return buf.value.decode()


class Batch:
    """Many independent CholeskyQR2 factorizations per call (cqr2_batch_*)."""

    def __init__(self, max_count: int, precision: int = CQR2_FP64, small_work_limit: int | None = None,
                 streams: int | None = None, fused: bool = True, stream=None, graph: bool = False):
        cfg = None
        if small_work_limit is not None or streams is not None or graph:
            cfg = N.BatchConfig(int(small_work_limit if small_work_limit is not None else 32768 * 64 * 64),
                                int(streams or 4), 1 if fused else 0, 1 if graph else 0)
        h = C.c_void_p()
        N.check(N.load().cqr2_batch_create(C.byref(h), int(max_count), precision,
                                           C.byref(cfg) if cfg is not None else None, _stream_handle(stream)),
                "cqr2_batch_create")
        self.handle = h
        self.max_count = int(max_count)

    class Descriptors:
        """A problem list's C descriptor array (see Batch.descriptors)."""

        def __init__(self, arr, count):
            self.arr, self.count = arr, count

    @staticmethod
    def descriptors(problems):
        """The C descriptor array of a problem list, reusable across factor()
        calls (the tensors must stay alive)."""
        k = len(problems)
        arr = (N.Problem * max(k, 1))()
        for i, pr in enumerate(problems):
            A, Q, R = pr[0], pr[1], pr[2]
            m, n = A.shape
            a, lda = _mat(A, m, n, "A")
            q, ldq = _mat(Q, m, n, "Q")
            r, ldr = _mat(R, n, n, "R")
            bp = xp = None
            if len(pr) > 3:
                bp, xp = _vec(pr[3], m, "b"), _vec(pr[4], n, "x")
            arr[i] = N.Problem(m, n, a, lda, q, ldq, r, ldr, bp, xp)
        return Batch.Descriptors(arr, k)

    def factor(self, problems, sync: bool = True):
        """problems: list of (A, Q, R) or, for least squares, (A, Q, R, b, x)
        with column-major CUDA float64 matrices and contiguous vectors b (m)
        and x (n), or the result of descriptors(). Returns a list of Info
        (sync=True) or None (then info() reports the outcomes)."""
        d = problems if isinstance(problems, Batch.Descriptors) else self.descriptors(problems)
        arr, k = d.arr, d.count
        infos = (Info * max(k, 1))() if sync else None
        st = N.load().cqr2_batch_factor(self.handle, arr, k, infos)
        self._last = k
        if st not in (CQR2_OK, CQR2_ERR_NOT_SPD):
            N.check(st, "cqr2_batch_factor")
        return list(infos)[:k] if sync else None

    def info(self):
        """Outcomes of the last factor() call (waits for it)."""
        k = getattr(self, "_last", 0)
        infos = (Info * max(k, 1))()
        st = N.load().cqr2_batch_info(self.handle, k, infos)
        if st not in (CQR2_OK, CQR2_ERR_NOT_SPD, N.CQR2_ERR_TIMEOUT):
            N.check(st, "cqr2_batch_info")
        return list(infos)[:k]

    def close(self) -> None:
        if getattr(self, "handle", None):
            N.load().cqr2_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ helpers

class Plan:
    """Owns a cqr2 plan for m x n factorizations on the current device."""

    def __init__(self, m: int, n: int, precision: int = CQR2_FP64, fused: bool = False, stream=None,
                 graph: bool = False, shifted: bool = False, inplace: bool = False):
        self.m, self.n = int(m), int(n)
        flags = ((CQR2_FUSED if fused else 0) | (N.CQR2_GRAPH if graph else 0) | (N.CQR2_SHIFTED if shifted else 0)
                 | (N.CQR2_INPLACE if inplace else 0))
        self.handle = cqr2_plan_create(self.m, self.n, precision, flags, stream)

    def factor_rows(self, A, Q=None, R=None, sync: bool = True):
        """Factor an m-row matrix with n <= m <= the plan's m."""
        m = A.shape[0]
        if Q is None:
            Q = empty_colmajor(m, self.n, device=A.device)
        if R is None:
            R = empty_colmajor(self.n, self.n, device=A.device)
        info = cqr2_factor_rows(self.handle, m, self.n, A, Q, R, sync)
        return Q, R, info

    def lstsq_rows(self, A, b, Q=None, R=None, x=None, sync: bool = True, keep_q: bool = True):
        """Least squares for an m-row matrix. With keep_q=False and no Q, Q
        goes to the plan's own buffer instead of a new tensor."""
        torch = _torch()
        m = A.shape[0]
        if Q is None and keep_q:
            Q = empty_colmajor(m, self.n, device=A.device)
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=A.device)
        info = cqr2_lstsq_rows(self.handle, m, self.n, A, b, x, Q, R, sync)
        return x, info

    def set_gram_ctas(self, ctas_per_sm: int) -> None:
        cqr2_plan_set_gram_ctas(self.handle, ctas_per_sm)

    def set_inverse_depth(self, depth: int) -> None:
        cqr2_plan_set_inverse_depth(self.handle, depth)

    def set_fused(self, fused: bool) -> None:
        cqr2_plan_set_fused(self.handle, fused)

    def set_panel_width(self, b: int) -> None:
        """Factor on column panels of width b (0 = plain CholeskyQR2)."""
        N.check(N.load().cqr2_plan_set_panel_width(self.handle, int(b)), "cqr2_plan_set_panel_width")

    def split_slices(self) -> int:
        """Slices per entry of the last factorization (0 native FP64; 6 or 7
        for a 6-slice plan, 7 when the device routed it to 7)."""
        v = C.c_int32(0)
        N.check(N.load().cqr2_plan_split_slices(self.handle, C.byref(v)), "cqr2_plan_split_slices")
        return int(v.value)

    def set_stream(self, stream) -> None:
        N.check(N.load().cqr2_plan_set_stream(self.handle, _stream_handle(stream)), "cqr2_plan_set_stream")

    @property
    def workspace_bytes(self) -> int:
        return cqr2_workspace_bytes(self.handle)

    def factor(self, A, Q=None, R=None, sync: bool = True):
        if Q is None:
            Q = empty_colmajor(self.m, self.n, device=A.device)
        if R is None:
            R = empty_colmajor(self.n, self.n, device=A.device)
        info = cqr2_factor(self.handle, self.m, self.n, A, Q, R, sync)
        return Q, R, info

    def lstsq(self, A, b, Q=None, R=None, x=None, sync: bool = True):
        torch = _torch()
        if Q is None:
            Q = empty_colmajor(self.m, self.n, device=A.device)
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=A.device)
        info = cqr2_lstsq(self.handle, self.m, self.n, A, b, x, Q, R, sync)
        return x, info

    def syrk(self, A, W=None):
        if W is None:
            W = empty_colmajor(self.n, self.n, device=A.device)
        cqr2_syrk(self.handle, self.m, self.n, A, W)
        return W

    def cholinv(self, W, L=None, Y=None, sync: bool = True):
        if L is None:
            L = empty_colmajor(self.n, self.n, device=W.device)
        if Y is None:
            Y = empty_colmajor(self.n, self.n, device=W.device)
        info = cqr2_cholinv(self.handle, self.n, W, L, Y, sync)
        return L, Y, info

    def qform(self, A, Rinv, Q=None):
        if Q is None:
            Q = empty_colmajor(self.m, self.n, device=A.device)
        cqr2_qform(self.handle, self.m, self.n, A, Rinv, Q)
        return Q

    def trmm_upper(self, R2, R1, R=None):
        if R is None:
            R = empty_colmajor(self.n, self.n, device=R1.device)
        cqr2_trmm_upper(self.handle, self.n, R2, R1, R)
        return R

    def factor_host(self, hA, hQ, hR) -> Info:
        return cqr2_factor_host(self.handle, self.m, self.n, hA, hQ, hR)

    def set_profiling(self, enable: bool) -> None:
        cqr2_plan_set_profiling(self.handle, enable)

    def stage_times(self) -> dict:
        return cqr2_plan_stage_times(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            cqr2_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def factor(A, fused: bool = False):
    """CholeskyQR2 of a column-major CUDA float64 matrix: returns (Q, R)."""
    A = colmajor(A)
    with Plan(A.shape[0], A.shape[1], fused=fused) as p:
        Q, R, _ = p.factor(A)
    return Q, R


def lstsq(A, b):
    """Least squares through CholeskyQR2: returns x."""
    A = colmajor(A)
    with Plan(A.shape[0], A.shape[1]) as p:
        x, _ = p.lstsq(A, b.contiguous())
    return x
