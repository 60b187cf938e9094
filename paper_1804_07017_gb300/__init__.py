"""Python binding of the GB300 LU library (``liblu_gb300.so``, C ABI in
``include/lu_gb300.h``).

The functions here carry the C entry points' names and only marshal
arguments: device pointers come from torch CUDA tensors (``data_ptr()``), the
stream from ``torch.cuda.current_stream()``.  Every step of the computation
runs in the library's CUDA kernels; when the library cannot be loaded every
call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from ._lib import (LU_ERR_CUDA, LU_ERR_HANDLE, LU_ERR_IO, LU_ERR_NOMEM, LU_ERR_TIMEOUT, LU_ERR_UNSUPPORTED,
                   LU_TUNE_F32, LU_TUNE_F64, LU_TUNE_BATCHED_F32, LU_TUNE_BATCHED_F64,
                   LU_F32, LU_F64, LU_SUCCESS, LU_TU_BF16, LU_TU_FP16, LU_TU_FP8, LU_TU_F32, LU_TU_BF16X3, LU_TU_BF16X6, LU_FULL_F64,
                   LU_WARN_NOT_CONVERGED, LuError, LuOpts, lib, library_path)
from .api import (Batch, Handle, lu_factor_batched, lu_gesv_batched, lu_solve_batched, default_opts, lu_factor, lu_factor_ex, lu_factor_mixed_ex, lu_gemm_update_ex, lu_gemm_update_tc_ex, lu_gesv_mixed, lu_laswp_ex,
                  lu_launch_count, lu_panel_factor_ex, lu_panel_factor_noalloc, lu_solve, lu_solve_ex, lu_trsm_ex,
                  lu_tune_clear, lu_tune_get, lu_tune_load, lu_tune_nb, lu_tune_save, lu_tune_set, lu_potrf_ex,
                  lu_tune_plan, lu_tune_plan_get, lu_step_trace, lu_step_trace_read, lu_geqrf_ex,
                  lu_potrf_mixed_ex, lu_geqrf_mixed_ex, lu_tune_batched)

__all__ = [
    "Batch", "Handle", "lu_factor_batched", "lu_gesv_batched", "lu_solve_batched", "LuError", "LuOpts", "default_opts", "lib", "library_path", "lu_factor", "lu_factor_ex",
    "lu_factor_mixed_ex", "lu_gemm_update_ex", "lu_gemm_update_tc_ex", "lu_gesv_mixed", "lu_laswp_ex", "lu_launch_count", "lu_panel_factor_ex", "lu_panel_factor_noalloc", "lu_solve",
    "lu_solve_ex", "lu_trsm_ex", "LU_F32", "LU_F64", "LU_SUCCESS", "LU_ERR_CUDA", "LU_ERR_HANDLE",
    "LU_ERR_NOMEM", "LU_ERR_TIMEOUT", "LU_ERR_UNSUPPORTED", "LU_WARN_NOT_CONVERGED", "LU_TU_BF16",
    "LU_TU_FP16", "LU_TU_FP8", "LU_TU_F32", "LU_TU_BF16X3", "LU_TU_BF16X6", "LU_FULL_F64",
    "LU_ERR_IO", "LU_TUNE_F64", "LU_TUNE_F32", "lu_tune_nb", "lu_tune_get", "lu_tune_set", "lu_tune_clear",
    "lu_tune_save", "lu_tune_load", "lu_potrf_ex", "lu_tune_plan", "lu_tune_plan_get", "lu_step_trace",
    "lu_step_trace_read", "lu_geqrf_ex", "lu_potrf_mixed_ex", "lu_geqrf_mixed_ex", "lu_tune_batched",
    "LU_TUNE_BATCHED_F64", "LU_TUNE_BATCHED_F32",
]
