"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/*.h, and rejects bad arguments with the
Level-3 BLAS argument positions before touching the device."""
import ctypes
import glob
import os
import re

import pytest

from paper_1912_04379_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        for m in re.finditer(r"GB_API\s+[\w\s\*]+?\b(gb_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_symbols()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(_lib.SIGNATURES) == names


def test_version_and_status_strings():
    lib = _lib.load()
    assert lib.gb_version() >= 10000
    for code in range(0, 8):
        assert lib.gb_status_string(code)
    assert b"argument" in lib.gb_status_string(-3)


BAD = [
    # (transa, transb, m, n, k, lda, ldb, ldc, expected)
    ("X", "N", 4, 4, 4, 4, 4, 4, -1),
    ("N", "Q", 4, 4, 4, 4, 4, 4, -2),
    ("N", "N", -1, 4, 4, 4, 4, 4, -3),
    ("N", "N", 4, -1, 4, 4, 4, 4, -4),
    ("N", "N", 4, 4, -1, 4, 4, 4, -5),
    ("N", "N", 5, 4, 4, 4, 4, 5, -8),     # lda < M
    ("T", "N", 5, 4, 6, 5, 6, 5, -8),     # lda < K for transposed A
    ("N", "N", 4, 4, 6, 4, 5, 4, -10),    # ldb < K
    ("N", "T", 4, 7, 6, 4, 6, 4, -10),    # ldb < N for transposed B
    ("N", "N", 6, 4, 4, 6, 4, 5, -13),    # ldc < M
    ("N", "N", 0, 0, 0, 0, 1, 1, -8),     # ld must be >= 1 even for empty matrices
]


@pytest.mark.parametrize("case", BAD, ids=[str(c[-1]) + "_" + c[0] + c[1] for c in BAD])
def test_blas_argument_codes(case):
    lib = _lib.load()
    ta, tb, m, n, k, lda, ldb, ldc, want = case
    rc = lib.gb_sgemm(None, 0, ta.encode(), tb.encode(), m, n, k, 1.0, None, lda, None, ldb, 0.0,
                      None, ldc, None, 0, None)
    assert rc == want
    out = ctypes.c_size_t()
    assert lib.gb_sgemm_workspace_size(1, ta.encode(), tb.encode(), m, n, k, ctypes.byref(out)) in (
        want, 0) or want in (-8, -10, -13)


def test_lowercase_and_conjugate_trans_accepted():
    lib = _lib.load()
    # valid arguments: with no handle the call fails on the handle, not on an argument
    for ta, tb in [("n", "t"), ("C", "c"), ("t", "N")]:
        rc = lib.gb_sgemm(None, 0, ta.encode(), tb.encode(), 3, 3, 3, 1.0, None, 3, None, 3, 0.0,
                          None, 3, None, 0, None)
        assert rc == _lib.GB_ERR_HANDLE


def test_workspace_sizes():
    lib = _lib.load()
    out = ctypes.c_size_t()
    assert lib.gb_sgemm_workspace_size(0, b"N", b"N", 100, 100, 100, ctypes.byref(out)) == 0
    assert out.value == 0                                    # SIMT needs none
    assert lib.gb_sgemm_workspace_size(2, b"N", b"N", 256, 128, 64, ctypes.byref(out)) == 0
    # BF16 x 2 terms: (256 + 128) rows * 64 k * 2 terms * 2 bytes
    assert out.value == (256 + 128) * 64 * 2 * 2
    assert lib.gb_sgemm_workspace_size(1, b"N", b"N", 256, 128, 64, ctypes.byref(out)) == 0
    assert out.value == (256 + 128) * 64 * 2 * 4             # TF32 words
    assert lib.gb_sgemm_workspace_size(3, b"T", b"N", 256, 128, 64, ctypes.byref(out)) == 0
    assert out.value == (256 + 128) * 64 * 3 * 2              # BF16 x 3 terms
    # rows of the packed terms start on 16-byte boundaries: k padded to 8 (BF16) / 4 (TF32)
    assert lib.gb_sgemm_workspace_size(2, b"N", b"N", 8, 8, 5, ctypes.byref(out)) == 0
    assert out.value == 2 * 1024                              # each region rounded to 1 KiB
    assert lib.gb_sgemm_workspace_size(2, b"N", b"N", 0, 8, 5, ctypes.byref(out)) == 0
    assert out.value == 0
    assert lib.gb_sgemm_workspace_size(7, b"N", b"N", 8, 8, 5, ctypes.byref(out)) == _lib.GB_ERR_ARG
    assert lib.gb_sgemm_workspace_size(2, b"N", b"N", 8, 8, 5, None) == _lib.GB_ERR_ARG


def test_backward_workspace_is_max_of_the_two_products():
    lib = _lib.load()
    out = ctypes.c_size_t()
    m, n, k = 64, 48, 32
    assert lib.gb_sgemm_backward_workspace_size(2, b"N", b"N", m, n, k, ctypes.byref(out)) == 0
    # dA: M x K x N product, dB: K x N x M product (BF16 x 2 terms, kpad rounds to 8)
    wa = 1024 * (-(-(m * n * 2 * 2) // 1024)) + 1024 * (-(-(k * n * 2 * 2) // 1024))
    wb = 1024 * (-(-(k * 64 * 2 * 2) // 1024)) + 1024 * (-(-(n * 64 * 2 * 2) // 1024))
    assert out.value == max(wa, wb)


def test_no_handle_without_gpu_or_bad_handle():
    lib = _lib.load()
    assert lib.gb_create(None) == _lib.GB_ERR_ARG
    assert lib.gb_destroy(None) == 0
    assert lib.gb_set_wait_limit(None, 10) == _lib.GB_ERR_HANDLE
    assert lib.gb_sgemm_grouped_destroy(None) == 0


def test_blas3_and_split_k_workspace_sizes():
    """Workspace sizes that follow from the library's layout rules, with no GPU:
    STRSM lays out every 256-row diagonal block's triangle and reciprocals
    (its 136 16 x 16 blocks on or below the diagonal, then 256 floats) after
    the GEMM updates' area
    (none for SIMT); BF16 x 3 terms keeps 256-column tiles for K > 2048, so a
    64 x 8192 output (32 tiles) with K = 8192 is cut into 4 K-slices of FP32
    partials, while at K = 2048 its 128-column tiles (64 of them) are enough."""
    lib = _lib.load()
    out = ctypes.c_size_t(0)
    simt = _lib.ALGOS["simt"]
    per_leaf = (16 * 17 // 2 * 16 * 16 + 256) * 4
    for side, uplo, tr, diag, m, n, leaves in (("L", "L", "N", "N", 300, 50, 2),
                                               ("R", "U", "T", "U", 10, 513, 3),
                                               ("L", "U", "N", "N", 256, 1, 1),
                                               ("L", "L", "N", "N", 0, 5, 0)):
        assert lib.gb_strsm_workspace_size(simt, side.encode(), uplo.encode(), tr.encode(),
                                           diag.encode(), m, n, ctypes.byref(out)) == 0
        assert out.value == leaves * per_leaf
    x6 = _lib.ALGOS["bf16x6"]
    packed = lambda rows, k: 3 * 2 * k * rows            # three BF16 terms, K padded to 8
    assert lib.gb_sgemm_workspace_size(x6, b"N", b"N", 64, 8192, 8192, ctypes.byref(out)) == 0
    assert out.value == packed(64, 8192) + packed(8192, 8192) + 4 * 64 * 8192 * 4
    assert lib.gb_sgemm_workspace_size(x6, b"N", b"N", 64, 8192, 2048, ctypes.byref(out)) == 0
    assert out.value == packed(64, 2048) + packed(8192, 2048)


def test_promotion_setting_arguments():
    """gb_set_promotion / gb_get_promotion validate their arguments without a
    device: a NULL handle is GB_ERR_HANDLE, a negative chunk GB_ERR_ARG."""
    lib = _lib.load()
    v = ctypes.c_int64(5)
    assert lib.gb_set_promotion(None, 64) == _lib.GB_ERR_HANDLE
    assert lib.gb_get_promotion(None, ctypes.byref(v)) == _lib.GB_ERR_HANDLE
    assert v.value == 5

