"""GPU checks specific to the scaled FP16 split (GB_ALGO_SPLIT_FP16X3).

Each row of op(A) and each block of 256 columns of op(B) is scaled by a
power of two chosen from its largest finite magnitude before the FP16
split, and the epilogue undoes it. Scaling a row (or a column block) by 2^s
therefore changes nothing but the exponent the kernel picks: the result
scales by exactly 2^s, bit for bit, as long as it stays in the normal FP32
range. The per-element
bound against the FP64 oracle is checked on rows and columns whose
magnitudes differ by up to 2^120, on empty (all-zero) rows, through the
pack-once path, and with and without promoted accumulation.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu import assert_within_bound, check_padding, oracle_of, run, torch_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    torch_gpu()
    import paper_1912_04379_gb300 as gb
    return gb.Handle()


def _scale_op_rows(X, trans, rows, s):
    """Multiply row i of op(X) (rows x k) by 2^s[i] in the stored matrix."""
    f = np.ldexp(np.float32(1.0), s).astype(np.float32)
    if trans == "N":
        X[:rows, :] *= f[:, None]
    else:
        X[:, :rows] *= f[None, :]


def _scale_op_cols(X, trans, cols, t):
    """Multiply column j of op(X) (k x cols) by 2^t[j] in the stored matrix."""
    f = np.ldexp(np.float32(1.0), t).astype(np.float32)
    if trans == "N":
        X[:, :cols] *= f[None, :]
    else:
        X[:cols, :] *= f[:, None]


@pytest.mark.parametrize("promote", (0, 64))
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_power_of_two_row_and_column_scaling_is_exact(h, ta, tb, promote):
    h.set_promotion(promote)
    m, n, k = 300, 600, 1500
    base = wl.make_problem(ta, tb, m, n, k, 1.0, 0.0, seed=61, ld_pad=3)
    rng = np.random.default_rng(62)
    s = rng.integers(-40, 41, m)
    t = np.repeat(rng.integers(-40, 41, 3), 256)[:n]     # one exponent per 256-column block
    scaled = wl.make_problem(ta, tb, m, n, k, 1.0, 0.0, seed=61, ld_pad=3)
    _scale_op_rows(scaled.A, ta, m, s)
    _scale_op_cols(scaled.B, tb, n, t)
    rc0, c0 = run(base, "fp16x3", handle=h)
    rc1, c1 = run(scaled, "fp16x3", handle=h)
    assert rc0 == 0 and rc1 == 0
    want = np.ldexp(c0[:m].astype(np.float64), s[:, None] + t[None, :])
    assert np.array_equal(c1[:m].astype(np.float64), want)
    assert_within_bound(scaled, c1, algo="fp16x3")
    h.set_promotion(0)


@pytest.mark.parametrize("promote", (0, 32))
def test_rows_and_columns_spanning_2_to_the_120(h, promote):
    h.set_promotion(promote)
    m, n, k = 257, 200, 700
    p = wl.make_problem("N", "T", m, n, k, -1.5, 0.25, seed=63, dist="logu", ld_pad=2)
    rng = np.random.default_rng(64)
    _scale_op_rows(p.A, "N", m, rng.integers(-60, 61, m))      # |op(A)| in [2^-80, 2^80]
    _scale_op_cols(p.B, "T", n, rng.integers(-10, 11, n))      # |op(B)| in [2^-30, 2^30]
    p.C[:m, :] = 0.0          # C's own magnitudes would dominate D otherwise
    rc, got = run(p, "fp16x3", handle=h)
    assert rc == 0
    assert_within_bound(p, got, algo="fp16x3")
    check_padding(p, got)
    h.set_promotion(0)


def test_zero_rows_and_columns(h):
    m, n, k = 200, 150, 333
    p = wl.make_problem("N", "N", m, n, k, 1.0, 0.5, seed=65, ld_pad=1)
    p.A[7, :] = 0.0
    p.A[130:140, :] = 0.0
    p.B[:, 3] = 0.0
    rc, got = run(p, "fp16x3", handle=h)
    assert rc == 0
    C = p.C[:m, :n].astype(np.float32)
    assert np.array_equal(got[7, :n], (np.float32(0.5) * C[7, :]))
    assert np.array_equal(got[130:140, 3], (np.float32(0.5) * C[130:140, 3]))
    assert_within_bound(p, got, algo="fp16x3")


def test_pack_and_compute_equal_gb_sgemm(h):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    h.set_promotion(64)
    m, n, k = 1100, 1300, 1500          # no split-K in gb_sgemm at this shape
    p = wl.make_problem("T", "N", m, n, k, 1.0, 0.0, seed=66, dist="logu")
    _, want = run(p, "fp16x3", handle=h)
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    C = gb.colmajor(m, n)
    Ap = torch.empty(gb.pack_size("fp16x3", "A", m, k), dtype=torch.uint8, device="cuda")
    Bp = torch.empty(gb.pack_size("fp16x3", "B", n, k), dtype=torch.uint8, device="cuda")
    kpad = (k + 7) // 8 * 8          # three FP16 terms for op(A), two for op(B), then the maxima
    assert Ap.numel() == (3 * m * kpad * 2 + 255) // 256 * 256 + 4 * m
    assert Bp.numel() == (2 * n * kpad * 2 + 255) // 256 * 256 + 4 * n
    gb.pack_raw("fp16x3", "A", "T", m, k, A.data_ptr(), p.lda, Ap, handle=h)
    gb.pack_raw("fp16x3", "B", "N", n, k, B.data_ptr(), p.ldb, Bp, handle=h)
    gb.compute_raw("fp16x3", m, n, k, 1.0, Ap, Bp, 0.0, C.data_ptr(), m, handle=h)
    torch.cuda.synchronize()
    assert np.array_equal(gb.to_fortran(C), want[:m])
    h.set_promotion(0)


def test_promotion_lowers_the_error_on_long_k(h):
    p = wl.split_case(256, 192, 8192, seed=2)
    C64, D = oracle_of(p)
    h.set_promotion(0)
    _, a = run(p, "fp16x3", handle=h)
    h.set_promotion(64)
    _, b = run(p, "fp16x3", handle=h)
    h.set_promotion(0)
    ra = oracle.err_report(a[:p.m], C64, D, p.k)
    rb = oracle.err_report(b[:p.m], C64, D, p.k)
    assert ra["max_ratio"] <= 1.0 and rb["max_ratio"] <= 1.0
    assert rb["max_ratio"] < ra["max_ratio"]
