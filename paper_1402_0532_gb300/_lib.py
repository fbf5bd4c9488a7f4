"""ctypes declarations of the C ABI in include/ndft.h (argument marshalling only).

Every function of the header is declared here under the same name.  Loading
fails loudly if libndft.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# NDFT_CHECKED=1 selects the index-checked build (libndft_checked.so), whose
# kernels test their global indices and report a failed test through the plan's
# error word
_CHECKED = os.environ.get("NDFT_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(_PKG, "libndft_checked.so" if _CHECKED else "libndft.so")

OK, E_INVALID, E_UNSUPPORTED, E_CUDA, E_NOMEM, E_TIMEOUT, E_OVERFLOW = range(7)
FORM_DIRECT, FORM_TERNARY_GEMM, FORM_NFFT, FORM_FFT = 0, 1, 2, 3
PREC_FP32, PREC_BF16X2, PREC_Q14 = 0, 1, 2
F_NO_CONJ_REF, F_CIRCULAR_LAG, F_NFFT_DIF, F_Q14_RANGE, F_ABS_OUT = 0x1, 0x2, 0x4, 0x8, 0x10

# every symbol include/ndft.h declares
EXPORTS = ("ndft_plan", "ndft_plan_batched", "ndft_plan_destroy", "ndft_exec", "nfft_exec", "caf_exec",
           "caf_exec_batched", "caf_backward", "caf_backward_inputs", "ndft_argmax", "ndft_query_error", "ndft_get_twiddles",
           "ndft_plan_bytes", "ndft_last_launches", "ndft_set_tuning", "ndft_timer_start", "ndft_timer_read",
           "ndft_status_string", "ndft_version", "ndft_last_cuda_error", "caf_exec_noalloc", "ndft_plan_query")


class NdftDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p0", ctypes.c_int32), ("nbins", ctypes.c_int32),
                ("max_lags", ctypes.c_int32), ("max_batch", ctypes.c_int64), ("form", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32 * 3)]


class NdftCpi(ctypes.Structure):
    _fields_ = [("off_surv", ctypes.c_int64), ("off_ref", ctypes.c_int64), ("off_out", ctypes.c_int64),
                ("n", ctypes.c_int32), ("lag0", ctypes.c_int32), ("nlags", ctypes.c_int32),
                ("p0", ctypes.c_int32), ("nbins", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class NdftError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        extra = ""
        if status in (E_CUDA, E_NOMEM) and _lib is not None:
            extra = f": {_lib.ndft_last_cuda_error().decode()}"
        super().__init__(f"{what}: {status_string(status)} (status {status}){extra}")


_lib = None


def load() -> ctypes.CDLL:
    """Load libndft.so (built by ``paper_1402_0532_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1402_0532_gb300.build.build() "
                          f"(checked={_CHECKED}; nvcc, sm_103a) before using the library; there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "ndft_plan": (i32, [ctypes.POINTER(P), ctypes.POINTER(NdftDesc), P]),
        "ndft_plan_batched": (i32, [ctypes.POINTER(P), ctypes.POINTER(NdftCpi), i32, i32, i32, u32, P]),
        "ndft_plan_destroy": (i32, [P]),
        "ndft_exec": (i32, [P, P, P, i64, P]),
        "nfft_exec": (i32, [P, P, P, i64, P]),
        "caf_exec": (i32, [P, P, P, i32, i32, P, P]),
        "caf_exec_batched": (i32, [P, P, P, P, P]),
        "caf_backward": (i32, [P, P, P, i32, i32, P, P, P]),
        "caf_backward_inputs": (i32, [P, P, P, i32, i32, P, P, P, P]),
        "ndft_argmax": (i32, [P, i64, i64, P, P, P]),
        "ndft_query_error": (i32, [P, P]),
        "ndft_get_twiddles": (i32, [P, i32, P, P]),
        "ndft_plan_bytes": (i32, [P, ctypes.POINTER(i64)]),
        "ndft_last_launches": (i32, [P, ctypes.POINTER(i32)]),
        "ndft_set_tuning": (i32, [P, i32, i32]),
        "ndft_plan_query": (i32, [P, i32, ctypes.POINTER(i64)]),
        "ndft_timer_start": (i32, [P, i32]),
        "ndft_timer_read": (i32, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]),
        "ndft_status_string": (ctypes.c_char_p, [i32]),
        "ndft_version": (i32, []),
        "ndft_last_cuda_error": (ctypes.c_char_p, []),
        "caf_exec_noalloc": (i32, [i32, i32, i32, P, P, i32, i32, u32, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().ndft_status_string(int(status)).decode()
    except ImportError:
        return "library not loaded"


def check(status: int, what: str):
    if status != OK:
        raise NdftError(status, what)
