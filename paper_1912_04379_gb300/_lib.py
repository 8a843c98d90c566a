"""ctypes declarations of the C ABI in include/gbsgemm.h (argument marshalling only).

The shared library is built in-tree by `paper_1912_04379_gb300.build`; if it
is missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p
c_f = ctypes.c_float
c_char = ctypes.c_char
c_int = ctypes.c_int
c_size = ctypes.c_size_t

ALGOS = {"auto": -1, "simt": 0, "tf32x3": 1, "bf16x3": 2, "bf16x6": 3, "bf16x9": 4, "fp16x3": 5}

GB_OK = 0
GB_ERR_CUDA = 1
GB_ERR_WORKSPACE = 2
GB_ERR_UNSUPPORTED = 3
GB_ERR_TIMEOUT = 4
GB_ERR_PLAN = 5
GB_ERR_HANDLE = 6
GB_ERR_ARG = 7


class ErrReport(ctypes.Structure):
    _fields_ = [("max_ratio", ctypes.c_double), ("median_ratio", ctypes.c_double),
                ("sum_sq_diff", ctypes.c_double), ("sum_sq_ref", ctypes.c_double),
                ("n_fail", c_i64), ("count", c_i64)]


class GemmProblem(ctypes.Structure):
    _fields_ = [("transa", c_char), ("transb", c_char), ("m", c_i64), ("n", c_i64), ("k", c_i64),
                ("alpha", c_f), ("beta", c_f), ("A", c_vp), ("lda", c_i64), ("B", c_vp),
                ("ldb", c_i64), ("C", c_vp), ("ldc", c_i64)]


class MlpDesc(ctypes.Structure):
    _fields_ = [("layers", c_i64), ("widths", ctypes.POINTER(c_i64)), ("batch", c_i64),
                ("hidden", c_int)]


ACTIVATIONS = {"identity": 0, "tanh": 1}

TUNING_MAX_GEMM = 64


class TuningGemm(ctypes.Structure):
    _fields_ = [("mode", c_int), ("log2_m", c_int), ("log2_n", c_int), ("log2_k", c_int),
                ("row_bytes", c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("gpu_name", ctypes.c_char * 96), ("sm_count", c_int),
                ("cuda_runtime_version", c_int), ("library_version", c_int),
                ("grouped_valid", c_int), ("grouped_route", c_int * 8), ("n_gemm", c_int),
                ("gemm", TuningGemm * TUNING_MAX_GEMM)]

SIGNATURES = {
    "gb_version": ([], c_int),
    "gb_status_string": ([c_int], ctypes.c_char_p),
    "gb_create": ([ctypes.POINTER(c_vp)], c_int),
    "gb_destroy": ([c_vp], c_int),
    "gb_sgemm_workspace_size": ([c_int, c_char, c_char, c_i64, c_i64, c_i64,
                                 ctypes.POINTER(c_size)], c_int),
    "gb_sgemm": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_i64, c_f, c_vp, c_i64, c_vp,
                  c_i64, c_f, c_vp, c_i64, c_vp, c_size, c_vp], c_int),
    "gb_sgemm_noalloc": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_i64, c_f, c_vp, c_i64,
                          c_vp, c_i64, c_f, c_vp, c_i64, c_vp], c_int),
    "gb_sgemm_pack_size": ([c_int, c_char, c_i64, c_i64, ctypes.POINTER(c_size)], c_int),
    "gb_sgemm_pack": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_vp, c_i64, c_vp, c_size,
                       c_vp], c_int),
    "gb_sgemm_compute": ([c_vp, c_int, c_i64, c_i64, c_i64, c_f, c_vp, c_vp, c_f, c_vp, c_i64,
                          c_vp], c_int),
    "gb_sgemm_backward": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_i64, c_f, c_vp, c_i64,
                           c_vp, c_i64, c_f, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64,
                           c_vp, c_size, c_vp], c_int),
    "gb_sgemm_backward_workspace_size": ([c_int, c_char, c_char, c_i64, c_i64, c_i64,
                                          ctypes.POINTER(c_size)], c_int),
    "gb_sgemm_grouped_plan": ([c_vp, c_int, c_i64, ctypes.POINTER(GemmProblem),
                               ctypes.POINTER(c_vp), ctypes.POINTER(c_size),
                               ctypes.POINTER(c_i64)], c_int),
    "gb_sgemm_grouped_run": ([c_vp, c_vp, c_size, c_vp], c_int),
    "gb_sgemm_grouped_destroy": ([c_vp], c_int),
    "gb_err_report_workspace_size": ([c_i64, c_i64], c_size),
    "gb_err_report": ([c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp,
                       c_size, ctypes.POINTER(ErrReport), c_vp], c_int),
    "gb_get_device_error": ([c_vp, c_vp, ctypes.POINTER(c_int)], c_int),
    "gb_set_wait_limit": ([c_vp, c_i64], c_int),
    "gb_set_fused_split": ([c_vp, c_int], c_int),
    "gb_set_skinny_split": ([c_vp, c_int], c_int),
    "gb_get_skinny_split": ([c_vp, ctypes.POINTER(c_int)], c_int),
    "gb_set_promotion": ([c_vp, c_i64], c_int),
    "gb_tune_grouped": ([c_vp], c_int),
    "gb_tune_sgemm": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_i64], c_int),
    "gb_get_tuning": ([c_vp, ctypes.POINTER(Tuning)], c_int),
    "gb_set_tuning": ([c_vp, ctypes.POINTER(Tuning)], c_int),
    "gb_tuning_write": ([ctypes.POINTER(Tuning), ctypes.c_char_p], c_int),
    "gb_tuning_read": ([ctypes.POINTER(Tuning), ctypes.c_char_p], c_int),
    "gb_get_promotion": ([c_vp, ctypes.POINTER(c_i64)], c_int),
    "gb_mlp_workspace_size": ([c_int, ctypes.POINTER(MlpDesc), c_int, ctypes.POINTER(c_size)],
                              c_int),
    "gb_mlp_forward": ([c_vp, c_int, ctypes.POINTER(MlpDesc), ctypes.POINTER(c_vp),
                        ctypes.POINTER(c_vp), c_vp, ctypes.POINTER(c_vp), c_vp, c_size, c_vp],
                       c_int),
    "gb_mlp_train_step": ([c_vp, c_int, ctypes.POINTER(MlpDesc), ctypes.POINTER(c_vp),
                           ctypes.POINTER(c_vp), c_vp, c_vp, c_f, ctypes.POINTER(c_vp),
                           ctypes.POINTER(c_vp), c_vp, c_vp, c_size, c_vp], c_int),
    "gb_sgemm_host_workspace_size": ([c_int, c_char, c_char, c_i64, c_i64, c_i64,
                                      ctypes.POINTER(c_size)], c_int),
    "gb_sgemm_host": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_i64, c_f, c_vp, c_i64, c_vp,
                       c_i64, c_f, c_vp, c_i64, c_vp, c_size, c_vp], c_int),
    "gb_measure_ffma": ([c_vp, c_i64, c_vp, ctypes.POINTER(c_i64), c_vp], c_int),
    "gb_ssyrk_workspace_size": ([c_int, c_char, c_char, c_i64, c_i64, ctypes.POINTER(c_size)],
                                c_int),
    "gb_ssyrk": ([c_vp, c_int, c_char, c_char, c_i64, c_i64, c_f, c_vp, c_i64, c_f, c_vp, c_i64,
                  c_vp, c_size, c_vp], c_int),
    "gb_strsm_workspace_size": ([c_int, c_char, c_char, c_char, c_char, c_i64, c_i64,
                                 ctypes.POINTER(c_size)], c_int),
    "gb_strsm": ([c_vp, c_int, c_char, c_char, c_char, c_char, c_i64, c_i64, c_f, c_vp, c_i64,
                  c_vp, c_i64, c_vp, c_size, c_vp], c_int),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgbsgemm.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} (run paper_1912_04379_gb300.build)")
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def status_string(code: int) -> str:
    return load().gb_status_string(int(code)).decode()


class GBError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn} returned {code}: {status_string(code)}")


def check(fn: str, code: int):
    if code != 0:
        raise GBError(fn, code)
