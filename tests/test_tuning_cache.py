"""The autotuning record's JSON cache (gb_tuning_write / gb_tuning_read):
host-only code, checked without a device. A record written and read back is
identical; malformed, truncated or missing files are refused with GB_ERR_ARG
and leave the output untouched; handle calls reject a NULL handle."""
import ctypes

import pytest

from paper_1912_04379_gb300 import _lib


def _record():
    t = _lib.Tuning()
    t.gpu_name = b"NVIDIA GB300 test"
    t.sm_count = 152
    t.cuda_runtime_version = 13000
    t.library_version = 10000
    t.grouped_valid = 1
    for c, v in enumerate((0, 0, 1, 2, 3, 4, 2, 3)):
        t.grouped_route[c] = v
    t.n_gemm = 3
    for i, (mode, lm, ln, lk, rb) in enumerate(((1, 13, 13, 13, 64), (2, 12, 12, 10, 128),
                                                 (4, 6, 13, 13, 64))):
        g = t.gemm[i]
        g.mode, g.log2_m, g.log2_n, g.log2_k, g.row_bytes = mode, lm, ln, lk, rb
    return t


def _fields(t):
    return (bytes(t.gpu_name), t.sm_count, t.cuda_runtime_version, t.library_version,
            t.grouped_valid, list(t.grouped_route), t.n_gemm,
            [(g.mode, g.log2_m, g.log2_n, g.log2_k, g.row_bytes) for g in t.gemm[:t.n_gemm]])


def test_round_trip(tmp_path):
    lib = _lib.load()
    path = str(tmp_path / "tuning.json").encode()
    t = _record()
    assert lib.gb_tuning_write(ctypes.byref(t), path) == 0
    r = _lib.Tuning()
    assert lib.gb_tuning_read(ctypes.byref(r), path) == 0
    assert _fields(r) == _fields(t)
    # and again: what was read writes the same file
    path2 = str(tmp_path / "again.json").encode()
    assert lib.gb_tuning_write(ctypes.byref(r), path2) == 0
    assert open(path, "rb").read() == open(path2, "rb").read()


def test_empty_gemm_table_round_trip(tmp_path):
    lib = _lib.load()
    t = _record()
    t.n_gemm = 0
    t.grouped_valid = 0
    path = str(tmp_path / "t.json").encode()
    assert lib.gb_tuning_write(ctypes.byref(t), path) == 0
    r = _lib.Tuning()
    assert lib.gb_tuning_read(ctypes.byref(r), path) == 0
    assert _fields(r) == _fields(t)


@pytest.mark.parametrize("damage", ["truncate", "format", "route", "missing"])
def test_bad_files_are_refused(tmp_path, damage):
    lib = _lib.load()
    path = tmp_path / "t.json"
    assert lib.gb_tuning_write(ctypes.byref(_record()), str(path).encode()) == 0
    text = path.read_text()
    if damage == "truncate":
        path.write_text(text[: len(text) // 2])
    elif damage == "format":
        path.write_text(text.replace("gbsgemm-tuning-1", "something-else"))
    elif damage == "route":
        path.write_text(text.replace('"grouped_route": [0, 0, 1', '"grouped_route": [0, 0'))
    else:
        path.unlink()
    r = _lib.Tuning()
    r.sm_count = -7
    assert lib.gb_tuning_read(ctypes.byref(r), str(path).encode()) == _lib.GB_ERR_ARG
    assert r.sm_count == -7                  # output untouched on failure


def test_handle_calls_need_a_handle():
    lib = _lib.load()
    t = _lib.Tuning()
    assert lib.gb_get_tuning(None, ctypes.byref(t)) == _lib.GB_ERR_HANDLE
    assert lib.gb_set_tuning(None, ctypes.byref(t)) == _lib.GB_ERR_HANDLE
    assert lib.gb_tune_grouped(None) == _lib.GB_ERR_HANDLE
    assert lib.gb_tune_sgemm(None, 2, b"N", b"N", 64, 64, 64) == _lib.GB_ERR_HANDLE
