"""The skinny-product kernel (one side at most 64 rows): the long operand
comes as FP32 by TMA and is split inside the kernel, the short one is packed,
the k-blocks are spread evenly over the SMs (stream-K) and a tile shared by
several SMs is summed by the last of them in slot order.

Checked against the FP64 oracle element by element (the product is the
SGEMM of paper Sec. 1 with the same split, so the same bound holds), with the
two-pass path (the switch off) beside it on the same inputs; integer data
bit-exact; repeated runs and graph replay bit-identical (the summation order
is fixed by the partition, not by timing); and that the kernel really runs
(its bits differ from the two-pass path's, and where the profiler records
kernels, its name is in the list)."""
import numpy as np
import pytest

import workloads as wl
from _gpu import (aligned_problem, assert_bit_exact, assert_within_bound, check_padding,
                  oracle_of, torch_gpu)

import oracle

pytestmark = pytest.mark.gpu
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]

# (m, n, k): short op(A) with a ragged last tile and k-block; a short side
# below 64 rows; short op(B); a single row; both sides 64 (one tile summed
# from every SM); long K over few tiles; many tiles with short K (most tiles
# shared by two SMs, many CTAs with a one-k-block first segment).
SHAPES = [(64, 3000, 1100), (37, 1500, 4099), (2000, 50, 2053), (1, 4096, 1030),
          (64, 64, 70000), (64, 8192, 640), (50, 20000, 300)]


@pytest.fixture(scope="module")
def handles():
    torch_gpu()
    import paper_1912_04379_gb300 as gb
    on, off = gb.Handle(), gb.Handle()
    assert on.skinny_split()
    off.set_skinny_split(False)
    assert not off.skinny_split()
    return on, off


def _run(p, algo, h, C=None):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    Cfull, _ = gb.from_fortran(p.C if C is None else C)
    assert A.data_ptr() % 16 == 0 and B.data_ptr() % 16 == 0
    gb.sgemm_raw(p.ta, p.tb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda, B.data_ptr(), p.ldb,
                 p.beta, Cfull.data_ptr(), p.ldc, algo=algo, handle=h)
    torch.cuda.synchronize()
    assert h.device_error() == (0, 0)
    return gb.to_fortran(Cfull)


def _kernel_names(fn):
    """Names of the CUDA kernels fn launched, from the profiler (skip when the
    profiler sees no kernels at all on this machine)."""
    torch = torch_gpu()
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    names = [e.name for e in prof.events() if "cuda" in str(e.device_type).lower()]
    if not names:
        pytest.skip("the profiler recorded no CUDA kernels")
    return names


@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6", "bf16x9"))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_skinny_within_bound(handles, algo, shape):
    on, off = handles
    m, n, k = shape
    i = SHAPES.index(shape)
    ta, tb = TRANS[i % 4]
    p = aligned_problem(ta, tb, m, n, k, 1.25, -0.5, seed=400 + i)
    got = _run(p, algo, on)
    ref = _run(p, algo, off)
    assert_within_bound(p, got, algo=algo)
    assert_within_bound(p, ref, algo=algo)
    check_padding(p, got)


@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6"))
def test_skinny_repeated_runs_identical(handles, algo):
    """Many tiles shared by two SMs, short K: 30 runs give the same bits and
    stay within the bound (a stage-reuse race showed here as stale rows)."""
    on, _ = handles
    p = aligned_problem("T", "N", 50, 20000, 300, 1.25, 0.0, seed=406)
    first = _run(p, algo, on)
    assert_within_bound(p, first, algo=algo)
    for _ in range(29):
        got = _run(p, algo, on)
        assert np.array_equal(got, first), f"{np.count_nonzero(got != first)} elements differ"


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6", "bf16x9"))
def test_skinny_all_transposes(handles, algo, ta, tb):
    on, _ = handles
    for (m, n, k) in ((40, 2100, 2500), (2100, 40, 2500)):
        p = aligned_problem(ta, tb, m, n, k, -0.75, 0.25, seed=m + 7 * k, dist="logu")
        got = _run(p, algo, on)
        assert_within_bound(p, got, algo=algo)
        check_padding(p, got)


@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6", "bf16x9"))
def test_skinny_integer_bit_exact(handles, algo):
    on, _ = handles
    for (ta, tb, m, n, k) in (("N", "N", 64, 4000, 4099), ("T", "T", 3000, 33, 3000)):
        p = aligned_problem(ta, tb, m, n, k, 1.0, 0.5, seed=17, dist="int")
        assert_bit_exact(p, _run(p, algo, on))


def test_skinny_beta_zero_does_not_read_c(handles):
    on, _ = handles
    p = aligned_problem("N", "N", 64, 3000, 2000, 1.0, 0.0, seed=18)
    C = p.C.copy(order="F")
    C[:p.m, :] = np.nan
    got = _run(p, "bf16x3", on, C=C)
    assert not np.isnan(got[:p.m]).any()
    assert_within_bound(p, got, algo="bf16x3")


def test_skinny_deterministic_and_graph_replay(handles):
    """Two eager runs and two replays of a captured call give the same bits."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    on, _ = handles
    p = aligned_problem("N", "N", 64, 8192, 2048, 1.0, 0.0, seed=19)
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    C, _ = gb.from_fortran(p.C)
    ws = torch.empty(gb.workspace_size("bf16x3", "N", "N", p.m, p.n, p.k), dtype=torch.uint8,
                     device="cuda")

    def call(stream=None):
        gb.sgemm_raw("N", "N", p.m, p.n, p.k, 1.0, A.data_ptr(), p.lda, B.data_ptr(), p.ldb,
                     0.0, C.data_ptr(), p.ldc, algo="bf16x3", handle=on, workspace=ws,
                     stream=stream)
    outs = []
    for _ in range(2):
        C.zero_()
        call()
        torch.cuda.synchronize()
        outs.append(C.clone())
    assert torch.equal(outs[0], outs[1])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            call(stream=s)
    torch.cuda.synchronize()
    for _ in range(2):
        C.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(C, outs[0])
    assert on.device_error() == (0, 0)


def test_skinny_kernel_is_the_one_that_runs(handles):
    """The switch decides the path: with it on, the skinny kernel's different
    summation order gives other bits than the two-pass path on random data;
    a leading dimension TMA cannot read (not a multiple of 4) falls back to
    the two-pass path, whose bits then equal the switched-off handle's. When
    the profiler records kernels, the kernel names confirm it."""
    on, off = handles
    p = aligned_problem("N", "N", 64, 4096, 2048, 1.0, 0.0, seed=20)
    got_on, got_off = _run(p, "bf16x3", on), _run(p, "bf16x3", off)
    assert not np.array_equal(got_on, got_off)
    assert_within_bound(p, got_on, algo="bf16x3")
    q = wl.make_problem("N", "N", 64, 4096, 2048, 1.0, 0.0, seed=21, ld_pad=1)
    q_on, q_off = _run(q, "bf16x3", on), _run(q, "bf16x3", off)
    assert np.array_equal(q_on, q_off)
    assert_within_bound(q, q_on, algo="bf16x3")
    try:
        names_on = _kernel_names(lambda: _run(p, "bf16x3", on))
    except pytest.skip.Exception:
        return
    assert any("tc_skinny_kernel" in x for x in names_on), names_on
    assert not any("tc_sgemm_kernel" in x for x in names_on), names_on
    names_q = _kernel_names(lambda: _run(q, "bf16x3", on))
    assert not any("tc_skinny_kernel" in x for x in names_q), names_q


def test_skinny_at_full_size_sampled(handles):
    """64 x 8192 x 8192 (the skinny bench shape), log-uniform magnitudes:
    sampled columns against the oracle within the plain FP32 bound."""
    on, _ = handles
    p = aligned_problem("N", "N", 64, 8192, 8192, 1.0, 0.0, seed=22, dist="logu")
    got = _run(p, "bf16x3", on)
    cols = np.unique(np.linspace(0, p.n - 1, 24).round().astype(np.int64))
    C64, D = oracle_of(p, cols=cols)
    rep = oracle.err_report(got[:p.m, cols], C64, D, p.k)
    assert rep["n_fail"] == 0 and rep["max_ratio"] <= 1.0, rep


def test_skinny_bounded_wait_expires_cleanly():
    """A 1 microsecond wait limit: every segment's accumulator takes far
    longer, so the epilogue's wait runs out; the status is reported, the CTAs
    drain their copies and MMAs, and the context still runs a correct GEMM."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.Handle()
    h.set_wait_limit(1)
    p = aligned_problem("N", "N", 64, 8192, 4096, 1.0, 0.0, seed=23)
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    C, _ = gb.from_fortran(p.C)
    gb.sgemm_raw("N", "N", p.m, p.n, p.k, 1.0, A.data_ptr(), p.lda, B.data_ptr(), p.ldb, 0.0,
                 C.data_ptr(), p.ldc, algo="bf16x3", handle=h)
    torch.cuda.synchronize()
    rc, site = h.device_error()
    assert rc == _lib.GB_ERR_TIMEOUT and site > 0
    h.set_wait_limit(2000000)
    q = aligned_problem("N", "N", 64, 3000, 1100, 1.0, 0.0, seed=24)
    got = _run(q, "bf16x3", h)
    assert_within_bound(q, got, algo="bf16x3")


def _vec_c_problem(ta, tb, m, n, k, alpha, beta, seed):
    """As aligned_problem, but C's leading dimension is a multiple of 4 (C
    rows 16-byte aligned): the float4 store path when op(A) is the short
    side."""
    p = aligned_problem(ta, tb, m, n, k, alpha, beta, seed)
    ldc = (m + 3) // 4 * 4 + 4
    C = wl.uniform(np.random.default_rng(seed + 1), m, n, ldc, pad=wl.CANARY)
    return wl.Problem(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.beta, p.A, p.lda, p.B, p.ldb, C,
                      C.shape[0])


@pytest.mark.parametrize("beta", (0.0, -0.5))
@pytest.mark.parametrize("m", (64, 50, 37))
def test_skinny_vector_c_stores(handles, m, beta):
    """C rows 16-byte aligned (ldc % 4 == 0): whole float4 stores, and a
    scalar tail when M is not a multiple of 4; beta != 0 reads C the same
    way. Both a whole-tile and a shared-tile (reduced) store occur (K long
    enough to split tiles over several CTAs)."""
    on, off = handles
    p = _vec_c_problem("N", "N", m, 6000, 3000, 1.25, beta, seed=300 + m)
    assert p.ldc % 4 == 0
    got = _run(p, "bf16x3", on)
    assert_within_bound(p, got, algo="bf16x3")
    check_padding(p, got)
    ref = _run(p, "bf16x3", off)
    assert_within_bound(p, ref, algo="bf16x3")


@pytest.mark.parametrize("shape", [(64, 8192, 255), (65, 8192, 2048), (100, 100, 100000)],
                         ids=lambda s: "x".join(map(str, s)))
def test_skinny_route_boundaries(handles, shape):
    """Just outside the skinny rule (K < 256; both sides over 64): the
    two-pass path runs whatever the switch says, so both handles give the
    same bits; both meet the bound."""
    on, off = handles
    m, n, k = shape
    p = aligned_problem("N", "N", m, n, k, 1.0, 0.0, seed=330 + m)
    a, b = _run(p, "bf16x6", on), _run(p, "bf16x6", off)
    assert np.array_equal(a, b)
    assert_within_bound(p, a, algo="bf16x6")
