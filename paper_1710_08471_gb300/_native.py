"""ctypes loader of libcqr2.so and raw signatures of the C ABI (include/cqr2.h).

There is no fallback: if the shared library is missing or cannot be loaded,
every call raises. Build it with ``paper_1710_08471_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libcqr2.so")

CQR2_OK = 0
CQR2_ERR_INVALID_ARG = 1
CQR2_ERR_NOT_SPD = 2
CQR2_ERR_CUDA = 3
CQR2_ERR_OOM = 4
CQR2_ERR_TIMEOUT = 5
CQR2_ERR_UNSUPPORTED = 6

CQR2_FP64 = 0
CQR2_OZAKI_BF16 = 1
CQR2_OZAKI_BF16_S6 = 2
CQR2_FUSED = 0x1
CQR2_GRAPH = 0x2
CQR2_SHIFTED = 0x4
CQR2_INPLACE = 0x8
CQR2_NUM_STAGES = 11


class Info(C.Structure):
    """cqr2_info_t"""
    _fields_ = [("status", C.c_int32), ("failed_pass", C.c_int32), ("failed_pivot", C.c_int64),
                ("pivot_value", C.c_double)]


class Problem(C.Structure):
    """cqr2_problem_t"""
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("A", C.c_void_p), ("lda", C.c_int64), ("Q", C.c_void_p),
                ("ldq", C.c_int64), ("R", C.c_void_p), ("ldr", C.c_int64), ("b", C.c_void_p), ("x", C.c_void_p)]


class BatchConfig(C.Structure):
    """cqr2_batch_config_t"""
    _fields_ = [("small_work_limit", C.c_int64), ("streams", C.c_int32), ("fused", C.c_int32), ("graph", C.c_int32)]


class TuneResult(C.Structure):
    """cqr2_tune_result_t"""
    _fields_ = [("gram_ctas", C.c_int32), ("fused", C.c_int32), ("ms", C.c_double), ("candidates", C.c_int32)]


_P = C.c_void_p
_D = C.c_void_p  # device pointer
_I64 = C.c_int64

# name -> (restype, argtypes); the single source of the binding's signatures.
SIGNATURES = {
    "cqr2_plan_create": (C.c_int, [C.POINTER(_P), _I64, _I64, C.c_int32, C.c_uint32, _P]),
    "cqr2_workspace_bytes": (C.c_size_t, [_P]),
    "cqr2_plan_set_stream": (C.c_int, [_P, _P]),
    "cqr2_plan_destroy": (None, [_P]),
    "cqr2_factor": (C.c_int, [_P, _D, _I64, _D, _I64, _D, _I64, C.POINTER(Info)]),
    "cqr2_lstsq": (C.c_int, [_P, _D, _I64, _D, _D, _D, _I64, _D, _I64, C.POINTER(Info)]),
    "cqr2_factor_rows": (C.c_int, [_P, _I64, _D, _I64, _D, _I64, _D, _I64, C.POINTER(Info)]),
    "cqr2_lstsq_rows": (C.c_int, [_P, _I64, _D, _I64, _D, _D, _D, _I64, _D, _I64, C.POINTER(Info)]),
    "cqr2_plan_info": (C.c_int, [_P, C.POINTER(Info)]),
    "cqr2_plan_split_slices": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "cqr2_plan_set_panel_width": (C.c_int, [_P, _I64]),
    "cqr2_plan_set_gram_ctas": (C.c_int, [_P, C.c_int32]),
    "cqr2_plan_set_fused": (C.c_int, [_P, C.c_int32]),
    "cqr2_plan_set_inverse_depth": (C.c_int, [_P, C.c_int32]),
    "cqr2_selftest_wait_timeout": (C.c_int, [C.c_int64, _P]),
    "cqr2_batch_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int32, C.POINTER(BatchConfig), _P]),
    "cqr2_batch_factor": (C.c_int, [_P, C.POINTER(Problem), C.c_int32, C.POINTER(Info)]),
    "cqr2_batch_info": (C.c_int, [_P, C.c_int32, C.POINTER(Info)]),
    "cqr2_autotune_batch": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(C.c_int64)]),
    "cqr2_batch_destroy": (None, [_P]),
    "cqr2_autotune": (C.c_int, [_I64, _I64, C.c_int32, C.POINTER(TuneResult)]),
    "cqr2_tune_set_small_limit": (C.c_int, [_I64]),
    "cqr2_tune_table": (C.c_int64, [C.c_char_p, _I64]),
    "cqr2_syrk": (C.c_int, [_P, _D, _I64, _D, _I64]),
    "cqr2_cholinv": (C.c_int, [_P, _D, _I64, _D, _I64, _D, _I64, C.POINTER(Info)]),
    "cqr2_qform": (C.c_int, [_P, _D, _I64, _D, _I64, _D, _I64]),
    "cqr2_trmm_upper": (C.c_int, [_P, _D, _I64, _D, _I64, _D, _I64]),
    "cqr2_syrk_noalloc": (C.c_int, [_D, _I64, _I64, _I64, _D, _I64, _P]),
    "cqr2_factor_host": (C.c_int, [_P, _P, _I64, _P, _I64, _P, _I64, C.POINTER(Info)]),
    "cqr2_plan_set_profiling": (C.c_int, [_P, C.c_int32]),
    "cqr2_plan_stage_times": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "cqr2_stage_name": (C.c_char_p, [C.c_int32]),
    "cqr2_launch_count": (C.c_int64, []),
    "cqr2_status_string": (C.c_char_p, [C.c_int]),
    "cqr2_version": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib: C.CDLL | None = None


def load(path: str | None = None) -> C.CDLL:
    """Load libcqr2.so (once) and attach the C signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libcqr2.so is not built ({p}); call paper_1710_08471_gb300.build.build()")
        lib = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class CQR2Error(RuntimeError):
    def __init__(self, status: int, where: str, info: Info | None = None):
        name = load().cqr2_status_string(status).decode()
        msg = f"{where}: {name}"
        if info is not None and status == CQR2_ERR_NOT_SPD:
            msg += f" (pass {info.failed_pass}, pivot {info.failed_pivot}, value {info.pivot_value!r})"
        super().__init__(msg)
        self.status = status
        self.info = info


def check(status: int, where: str, info: Info | None = None) -> None:
    if status != CQR2_OK:
        raise CQR2Error(status, where, info)
