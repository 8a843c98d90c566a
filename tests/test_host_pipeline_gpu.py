"""gb_sgemm_host (host buffers, copies pipelined with the GEMM on the handle's
streams) against the FP64 oracle: per-element bound of the algorithm, the
padding rows of the host C untouched, C not read when beta = 0, bit-exact on
integer data, and ordering on the caller's stream."""
import numpy as np
import pytest

import workloads as wl
from _gpu import assert_bit_exact, assert_within_bound, auto_algo, check_padding, torch_gpu

pytestmark = pytest.mark.gpu
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


def _pinned(arr):
    """A pinned torch tensor holding the Fortran array's storage (column-major)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(arr, dtype=np.float32).T)).pin_memory()


def _run_host(p, algo, stream=None):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    A, B, C = _pinned(p.A), _pinned(p.B), _pinned(p.C)
    gb.sgemm_host_raw(p.ta, p.tb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda, B.data_ptr(),
                      p.ldb, p.beta, C.data_ptr(), p.ldc, algo=algo, stream=stream)
    (stream or torch.cuda.current_stream()).synchronize()
    return np.asfortranarray(C.numpy().T)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("shape", [(300, 1000, 200), (130, 2600, 1100), (1, 1, 1), (517, 300, 70)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("algo", ("simt", "bf16x6", "auto"))
def test_host_pipeline_against_oracle(algo, shape, ta, tb):
    m, n, k = shape
    p = wl.make_problem(ta, tb, m, n, k, 1.25, -0.5, seed=m + n + k, ld_pad=3)
    got = _run_host(p, algo)
    if algo == "auto":
        algo = auto_algo(k)
    assert_within_bound(p, got, algo=algo)
    check_padding(p, got)


@pytest.mark.parametrize("algo", ("tf32x3", "bf16x3", "bf16x9", "fp16x3"))
def test_host_pipeline_splits(algo):
    p = wl.make_problem("T", "N", 260, 1800, 1500, -0.75, 0.0, seed=81, dist="logu", ld_pad=1)
    p.C[:p.m, :] = np.nan                      # beta = 0: C is not read
    got = _run_host(p, algo)
    assert_within_bound(p, got, algo=algo)
    check_padding(p, got)


def test_host_pipeline_integer_bit_exact():
    p = wl.make_problem("N", "T", 333, 2000, 1200, 1.0, 0.5, seed=82, dist="int", ld_pad=2)
    assert_bit_exact(p, _run_host(p, "auto"))


def test_host_pipeline_scale_only_and_quick_return():
    p = wl.make_problem("N", "N", 200, 700, 50, 0.0, -2.0, seed=83, ld_pad=1)
    p.A[:] = np.nan
    p.B[:] = np.nan
    got = _run_host(p, "auto")
    assert np.array_equal(got[:p.m, :], np.float32(-2.0) * p.C[:p.m, :])
    check_padding(p, got)
    p1 = wl.make_problem("N", "N", 20, 30, 0, 1.0, 1.0, seed=84)
    assert np.array_equal(_run_host(p1, "auto"), p1.C)


def test_host_pipeline_is_ordered_on_the_callers_stream():
    """Work enqueued on the stream before the call finishes first (a device
    copy into the pinned A), and the stream waits for the call's last copy."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, n, k = 256, 1500, 300
    p = wl.make_problem("N", "N", m, n, k, 1.0, 0.0, seed=85)
    A, B, C = _pinned(p.A), _pinned(p.B), _pinned(p.C)
    s = torch.cuda.Stream()
    src = torch.from_numpy(np.ascontiguousarray(p.A.T)).cuda()
    A.zero_()
    with torch.cuda.stream(s):
        A.copy_(src, non_blocking=True)          # enqueued before the GEMM on s
        gb.sgemm_host_raw("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0,
                          C.data_ptr(), m, algo="bf16x6", stream=s)
        done = torch.cuda.Event()
        done.record(s)
    done.synchronize()
    assert_within_bound(p, np.asfortranarray(C.numpy().T), algo="bf16x6")


def test_host_pipeline_argument_errors():
    torch_gpu()
    import paper_1912_04379_gb300 as gb
    assert gb.sgemm_host_raw("X", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4, check=False) == -1
    assert gb.sgemm_host_raw("N", "N", 4, 4, 4, 1.0, 0, 3, 0, 4, 0.0, 0, 4, check=False) == -8
    assert gb.sgemm_host_raw("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 3, check=False) == -13


# ---- the 2-D blocked pipeline (split algorithms, M and N >= 2048): op(A) row
# blocks and op(B) column blocks of 1024 (ragged last ones), unequal counts

SHAPES_2D = [(2100, 2300, 700), (4100, 2048, 300), (2048, 5000, 1500)]


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("shape", SHAPES_2D, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("algo", ("bf16x6", "fp16x3", "auto"))
def test_host_pipeline_2d_against_oracle(algo, shape, ta, tb):
    m, n, k = shape
    p = wl.make_problem(ta, tb, m, n, k, 1.25, -0.5, seed=m + 3 * n + k, ld_pad=3)
    got = _run_host(p, algo)
    if algo == "auto":
        algo = "bf16x3" if k >= 1024 else "bf16x6"
    # every block boundary of C and its neighbours, plus a spread of columns
    cols = np.unique(np.r_[0, 1, np.arange(1023, n, 1024), np.arange(1024, n, 1024),
                           np.linspace(0, n - 1, 24).round().astype(int), n - 1])
    cols = cols[cols < n]
    assert_within_bound(p, got, cols=cols, algo=algo)
    check_padding(p, got)


@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6", "fp16x3"))
def test_host_pipeline_2d_equals_device_gemm(algo):
    """K > 2048: the blocked GEMMs run the same kernel configuration as one
    gb_sgemm over the whole shape (which has enough tiles not to split K),
    and an output element's arithmetic does not depend on its tile, so the
    results agree bit for bit; beta = 0 with NaN in C (not read)."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from _gpu import run
    p = wl.make_problem("N", "T", 2100, 2300, 2500, 1.0, 0.0, seed=86, dist="logu", ld_pad=1)
    p.C[:p.m, :] = np.nan
    got = _run_host(p, algo)
    _, want = run(p, algo)
    assert np.array_equal(got[:p.m], want[:p.m])
    check_padding(p, got)


def test_host_pipeline_2d_integer_bit_exact_beta():
    p = wl.make_problem("T", "N", 3000, 2200, 900, 1.0, -0.5, seed=87, dist="int", ld_pad=2)
    assert_bit_exact(p, _run_host(p, "bf16x6"))
