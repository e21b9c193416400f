"""Thin ctypes binding of the C ABI in include/core_als.h.

Every function here only marshals arguments: it takes torch CUDA tensors (or
raw integers for pointers), passes their device addresses and sizes to the
library, and turns a negative status into an exception. All arithmetic runs
in the CUDA kernels of libcore_als.so; there is no CPU fallback. Loading
fails with an error when the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

from . import build as _build

ALS_OK = 0
STATUS = {
    0: "ALS_OK", -1: "ALS_ERR_ARG", -2: "ALS_ERR_CSR", -3: "ALS_ERR_NONFINITE", -4: "ALS_ERR_CUDA",
    -5: "ALS_ERR_TIMEOUT", -6: "ALS_ERR_OOM", -7: "ALS_ERR_DEVICE_BOUNDS", -8: "ALS_ERR_UNSUPPORTED",
}
ALS_REG_WEIGHTED, ALS_REG_PLAIN = 0, 1
ALS_GRAM_ASYM, ALS_GRAM_SYM, ALS_GRAM_FULL = 0, 1, 2
ALS_FP32, ALS_TF32, ALS_BF16, ALS_FP32_TC = 0, 1, 2, 3
ALS_FLAG_RATIO, ALS_FLAG_SINGULAR, ALS_FLAG_FP64 = 1, 2, 4
ALS_REFINE_AUTO = -1
ALS_SKETCH_SLICE, ALS_SKETCH_FACTOR = 0, 1
PROBES = {"ffma": 0, "dfma": 1, "tc_bf16": 2, "tc_tf32": 3, "l2_gather": 4, "hbm_copy": 5}
ALS_SSE_STATIC_MAX_ENTRIES = 4096 * 16384


class AlsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class als_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("indptr", C.c_void_p), ("indices", C.c_void_p), ("values", C.c_void_p)]


class als_options(C.Structure):
    _fields_ = [("n_f", C.c_int), ("lambda_", C.c_float), ("budget", C.c_double), ("min_keep", C.c_int64),
                ("reg_mode", C.c_int), ("gram_mode", C.c_int), ("precision", C.c_int),
                ("pivot_ratio_max", C.c_double), ("fp64_fallback", C.c_int), ("refine_steps", C.c_int),
                ("fixed_keep", C.c_int64), ("sketch", C.c_int)]


class als_report(C.Structure):
    _fields_ = [("rows_flagged", C.c_int64), ("rows_singular", C.c_int64), ("rows_fp64", C.c_int64),
                ("max_pivot_ratio", C.c_double),
                ("test_rmse", C.c_double), ("objective", C.c_double), ("sweeps_done", C.c_int)]


class als_tuning(C.Structure):
    _fields_ = [("split_at_middle", C.c_int), ("warp_rows", C.c_int), ("tc_gram", C.c_int),
                ("ms_per_sweep", C.c_double)]


class als_problem(C.Structure):
    _fields_ = [("users", als_csr), ("items", als_csr), ("n_f", C.c_int), ("U", C.c_void_p), ("M", C.c_void_p)]


# Every symbol the header declares, with (restype, argtypes).
_P = C.c_void_p
_I64 = C.c_int64
SIGNATURES = {
    "als_default_options": (None, [_P]),
    "als_create": (C.c_int, [_P, _P, _P]),
    "als_destroy": (C.c_int, [_P]),
    "als_set_stream": (C.c_int, [_P, _P]),
    "als_get_options": (C.c_int, [_P, _P]),
    "als_prepare": (C.c_int, [_P, _P]),
    "als_half_sweep": (C.c_int, [_P, _P, _P, _P, _P]),
    "als_select": (C.c_int, [_P, _P, _P, _P]),
    "als_assemble": (C.c_int, [_P, _P, _P, _P, _P]),
    "als_solve": (C.c_int, [_P, _I64, _P, _P, _P, _P]),
    "als_eval_sse": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P]),
    "als_eval_sse_async": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P]),
    "als_eval_sse_static": (C.c_int, [_I64, _P, _P, _P, _P, _P, C.c_int, _P, _P]),
    "als_objective": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "als_eval_remse": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P]),
    "als_eval_ranking": (C.c_int, [_P, _P, _P, _P, _P, C.c_int, C.c_int, _P, _P, _P, _P]),
    "als_profile": (C.c_int, [_P, C.c_int]),
    "als_kernel_time": (C.c_int, [_P, C.c_char_p, _P, _P]),
    "als_get_report": (C.c_int, [_P, _P]),
    "als_wait_selftest": (C.c_int, [_P, C.c_int64, C.c_int]),
    "als_sweep": (C.c_int, [_P, _P, _P, _P, _P]),
    "als_fit": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _I64, _P, _P, _P, _P]),
    "als_fit_host": (C.c_int, [_P, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P, _I64, _P, _P,
                               _P, _P]),
    "als_autotune": (C.c_int, [_P, _P, _P, _P, _P, C.c_int, _P]),
    "als_set_tuning": (C.c_int, [_P, _P]),
    "als_get_tuning": (C.c_int, [_P, _P]),
    "als_batch_create": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "als_batch_fit": (C.c_int, [_P, C.c_int]),
    "als_batch_select": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "als_batch_launches_per_sweep": (_I64, [_P]),
    "als_batch_destroy": (C.c_int, [_P]),
    "als_features": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "als_mlp_create": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_uint64, _P]),
    "als_mlp_destroy": (C.c_int, [_P]),
    "als_mlp_num_params": (_I64, [_P]),
    "als_mlp_set_params": (C.c_int, [_P, _P]),
    "als_mlp_get_params": (C.c_int, [_P, _P]),
    "als_mlp_forward": (C.c_int, [_P, _I64, _P, _P]),
    "als_mlp_grad": (C.c_int, [_P, _I64, _P, _P, _P, _P]),
    "als_mlp_train_step": (C.c_int, [_P, _I64, _P, _P, C.c_float, _P]),
    "als_probe": (C.c_int, [C.c_int, _P, _P, _P]),
    "als_workspace_bytes": (_I64, [_P]),
    "als_launch_count": (_I64, [_P]),
    "als_status_string": (C.c_char_p, [C.c_int]),
    "als_last_error": (C.c_char_p, [_P]),
}

_lib = None


def library_path() -> Path:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcore_als.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not path.exists():
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_2509_18024_gb300.build.build()")
        _build.build()
    lib = C.CDLL(str(path))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, handle=None):
    if status != ALS_OK:
        lib = load()
        msg = lib.als_last_error(handle).decode() if handle else lib.als_status_string(status).decode()
        raise AlsError(status, msg)


def ptr(t) -> int | None:
    """Device address of a tensor (None for None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()
