"""ctypes loader for liblu_gb300.so and the C ABI's signatures."""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(_HERE, "..", "include", "lu_gb300.h")

LU_SUCCESS = 0
LU_ERR_CUDA = -101
LU_ERR_NOMEM = -102
LU_ERR_TIMEOUT = -103
LU_ERR_UNSUPPORTED = -104
LU_ERR_HANDLE = -105
LU_ERR_IO = -106
LU_WARN_NOT_CONVERGED = 0x40000000

LU_F64 = 0
LU_F32 = 1

KERNEL_CLASSES = ["panel", "laswp", "trsm", "gemm", "tc_update", "pack", "solve", "residual", "other", "batched"]

LU_TU_BF16 = 0
LU_TU_FP16 = 1
LU_TU_FP8 = 2
LU_TU_F32 = 3
LU_TU_BF16X3 = 4
LU_FULL_F64 = 5
LU_TU_BF16X6 = 6

LU_TUNE_F64 = 100
LU_TUNE_F32 = 101
LU_TUNE_BATCHED_F64 = 102
LU_TUNE_BATCHED_F32 = 103


class LuError(RuntimeError):
    def __init__(self, name: str, code: int, detail: str = ""):
        super().__init__(f"{name} returned {code}" + (f": {detail}" if detail else ""))
        self.code = code


class LuOpts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("lookahead", ctypes.c_int), ("steal", ctypes.c_int),
                ("leaf", ctypes.c_int), ("pf_ctas", ctypes.c_int), ("tu_reserve", ctypes.c_int),
                ("nsched", ctypes.c_int), ("sched", ctypes.POINTER(ctypes.c_int32)), ("rtm", ctypes.c_int),
                ("pf_sms", ctypes.c_int)]

    def set_schedule(self, widths):
        """Per-step block sizes (kept alive with the options); None or [] clears."""
        if not widths:
            self._sched_buf = None
            self.nsched = 0
            self.sched = None
            return self
        self._sched_buf = (ctypes.c_int32 * len(widths))(*[int(w) for w in widths])
        self.nsched = len(widths)
        self.sched = ctypes.cast(self._sched_buf, ctypes.POINTER(ctypes.c_int32))
        return self

    def schedule(self):
        return [int(self.sched[i]) for i in range(self.nsched)] if self.nsched > 0 else []


def library_path() -> str:
    return os.environ.get("LU_GB300_LIB", os.path.join(_HERE, "liblu_gb300.so"))


i64, i32, vp, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
_SIGNATURES = {
    "lu_default_opts": (None, [ctypes.POINTER(LuOpts)]),
    "lu_create": (i32, [ctypes.POINTER(vp)]),
    "lu_destroy": (i32, [vp]),
    "lu_set_stream": (i32, [vp, vp]),
    "lu_launch_count": (i64, []),
    "lu_last_error": (ctypes.c_char_p, []),
    "lu_factor": (i32, [i64, vp, i64, vp, i32]),
    "lu_solve": (i32, [i64, i64, vp, vp, vp]),
    "lu_factor_ex": (i32, [vp, i32, i64, vp, i64, vp, ctypes.POINTER(LuOpts), vp]),
    "lu_solve_ex": (i32, [vp, i32, i64, i64, vp, i64, vp, vp, i64]),
    "lu_panel_factor_ex": (i32, [vp, i32, i64, i64, vp, i64, vp, ctypes.POINTER(LuOpts), vp]),
    "lu_laswp_ex": (i32, [vp, i32, i64, vp, i64, i64, i64, vp]),
    "lu_trsm_ex": (i32, [vp, i32, i64, i64, vp, i64, vp, i64]),
    "lu_gemm_update_ex": (i32, [vp, i32, i64, i64, i64, vp, i64, vp, i64, vp, i64]),
    "lu_gemm_update_tc_ex": (i32, [vp, i32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]),
    "lu_panel_factor_noalloc": (i32, [i32, i64, i64, vp, i64, vp, ctypes.POINTER(LuOpts), vp, vp]),
    "lu_noalloc_scratch_bytes": (ctypes.c_size_t, []),
    "lu_selftest_wait_timeout": (i32, [vp, i64, vp]),
    "lu_peak_fma": (i32, [i32, i32, i32, i64, vp, vp]),
    "lu_peak_fma_chains": (i32, []),
    "lu_profile_enable": (i32, [i32]),
    "lu_profile_stride": (i32, [i32]),
    "lu_profile_reset": (i32, []),
    "lu_profile_read": (i32, [i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                              ctypes.POINTER(dbl)]),
    "lu_gesv_batched": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
    "lu_factor_batched": (i32, [vp, i32, i32, vp, vp, vp, vp, vp]),
    "lu_solve_batched": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
    "lu_factor_mixed_ex": (i32, [vp, i32, i64, vp, i64, vp, ctypes.POINTER(LuOpts), vp]),
    "lu_gesv_mixed": (i32, [vp, i32, i64, i64, vp, i64, vp, i64, vp, i64, dbl, i32, ctypes.POINTER(LuOpts),
                            ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
    "lu_potrf_ex": (i32, [vp, i32, i64, vp, i64, ctypes.POINTER(LuOpts), vp]),
    "lu_tune_nb": (i32, [vp, i32, i64, ctypes.POINTER(i32), i32, i32, ctypes.POINTER(LuOpts), ctypes.POINTER(i32),
                         ctypes.POINTER(ctypes.c_float)]),
    "lu_tune_get": (i32, [ctypes.c_char_p, i32, i64]),
    "lu_tune_set": (i32, [ctypes.c_char_p, i32, i64, i32, ctypes.c_float]),
    "lu_tune_clear": (i32, []),
    "lu_tune_save": (i32, [ctypes.c_char_p]),
    "lu_tune_load": (i32, [ctypes.c_char_p]),
    "lu_tune_plan": (i32, [vp, i32, i64, i32, ctypes.POINTER(LuOpts), ctypes.POINTER(LuOpts),
                           ctypes.POINTER(ctypes.c_int32), i32, ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(ctypes.c_float)]),
    "lu_tune_plan_set": (i32, [ctypes.c_char_p, i32, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_int32), i32,
                               i32, ctypes.c_float]),
    "lu_tune_plan_get": (i32, [ctypes.c_char_p, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int32), i32, ctypes.POINTER(i32),
                               ctypes.POINTER(i32)]),
    "lu_geqrf_ex": (i32, [vp, i32, i64, i64, vp, i64, vp, ctypes.POINTER(LuOpts), vp]),
    "lu_potrf_mixed_ex": (i32, [vp, i32, i64, vp, i64, ctypes.POINTER(LuOpts), vp]),
    "lu_geqrf_mixed_ex": (i32, [vp, i32, i64, i64, vp, i64, vp, ctypes.POINTER(LuOpts), vp]),
    "lu_tune_batched": (i32, [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), i32, ctypes.POINTER(i32), i32,
                              ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]),
    "lu_step_trace": (i32, [vp, i32]),
    "lu_step_trace_read": (i64, [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float)]),
}

_lib = None


def lib():
    """Load the library (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise OSError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols(header: str = HEADER) -> list[str]:
    """Function names declared in the public header."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lu_[a-z0-9_]+)\s*\(", text)))


def signatures() -> dict:
    return dict(_SIGNATURES)
