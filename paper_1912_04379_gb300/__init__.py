"""GB300 (sm_103a) single-precision GEMM: C <- alpha*op(A)*op(B) + beta*C.

The computation of Aberdeen & Baxter's Emmerald SGEMM (Level-3 BLAS SGEMM,
paper Sec. 1), re-designed for the GB300: a plain FP32 SIMT kernel and
split-precision tensor-core kernels (tcgen05/TMEM/TMA) behind the C ABI in
include/gbsgemm.h. This package is the thin Python binding: importing it
does not load the CUDA library; the first call does, and fails loudly if
the library is missing.
"""
from .api import (GroupedPlan, Handle, backward_raw, colmajor, compute_raw, default_handle,
                  err_report, from_fortran, pack_raw, pack_size, sgemm, sgemm_host_raw,
                  sgemm_host_workspace_size, sgemm_raw, ssyrk_raw, strsm_raw, to_fortran,
                  upload_problems, workspace_size)
from .mlp import MLP

__all__ = ["MLP", "GroupedPlan", "Handle", "backward_raw", "colmajor", "compute_raw",
           "default_handle", "err_report", "from_fortran", "pack_raw", "pack_size", "sgemm",
           "sgemm_host_raw", "sgemm_host_workspace_size", "sgemm_raw", "ssyrk_raw", "strsm_raw", "to_fortran", "upload_problems",
           "workspace_size"]
