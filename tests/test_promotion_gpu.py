"""GPU parity of promoted accumulation (gb_set_promotion), through the C ABI.

The tensor cores' FP32 accumulation truncates; with promotion the kernel
starts a fresh tensor-memory accumulator every k_chunk elements of K and
adds the chunks on the CUDA cores in FP32 round-to-nearest. The product is
still the SGEMM of paper Sec. 1, so every element must meet the same bound
against the FP64 oracle, integer data stay bit-exact, and with one chunk
covering all of K the result must equal the unpromoted kernel's bit for bit
(same k-blocks, same MMA order, same epilogue arithmetic) wherever that
kernel runs the same tile configuration (64-byte rows: K > 2048, or the
two-term splits with K > 128).
"""
import numpy as np
import pytest

import workloads as wl
from _gpu import assert_bit_exact, assert_within_bound, check_padding, oracle_of, run, torch_gpu

import oracle

pytestmark = pytest.mark.gpu
SPLIT = ("tf32x3", "bf16x3", "bf16x6", "bf16x9", "fp16x3")
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


@pytest.fixture(scope="module")
def handles():
    torch_gpu()
    import paper_1912_04379_gb300 as gb
    return gb.Handle(), gb.Handle()


def _promoted(h, kc):
    h.set_promotion(kc)
    assert h.promotion() == kc
    return h


@pytest.mark.parametrize("algo", SPLIT)
@pytest.mark.parametrize("shape", [(1000, 1300, 2100), (300, 520, 2100), (129, 257, 4099),
                                   (64, 1000, 4096)],
                         ids=lambda s: "x".join(map(str, s)))
def test_one_chunk_is_bit_identical_to_the_plain_kernel(handles, algo, shape):
    """k_chunk >= K: one chunk per tile (or per split-K slice: every shape
    here but the first splits K), so the promoted kernel must reproduce the
    plain one exactly."""
    plain, promo = handles
    plain.set_promotion(0)
    _promoted(promo, 1 << 20)
    m, n, k = shape
    for ta, tb in (("N", "N"), ("T", "T")):
        p = wl.make_problem(ta, tb, m, n, k, 1.25, -0.5, seed=80 + m, ld_pad=3)
        rc0, want = run(p, algo, handle=plain)
        rc1, got = run(p, algo, handle=promo)
        assert rc0 == 0 and rc1 == 0
        assert np.array_equal(got, want), \
            f"{np.count_nonzero(got != want)} elements differ from the plain kernel"
    assert promo.device_error() == (0, 0)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("kc", (1, 32, 64, 256))
@pytest.mark.parametrize("algo", SPLIT)
def test_promoted_within_bound(handles, algo, kc, ta, tb):
    _, h = handles
    _promoted(h, kc)
    for (m, n, k) in ((257, 300, 1000), (130, 513, 77), (33, 7, 2049)):
        p = wl.make_problem(ta, tb, m, n, k, 1.5, -0.5, seed=90 + k, ld_pad=5)
        rc, got = run(p, algo, handle=h)
        assert rc == 0
        assert_within_bound(p, got, algo=algo)
        check_padding(p, got)
    assert h.device_error() == (0, 0)


@pytest.mark.parametrize("kc", (32, 96))
@pytest.mark.parametrize("algo", SPLIT)
def test_promoted_integer_bit_exact(handles, algo, kc):
    _, h = handles
    _promoted(h, kc)
    for (m, n, k) in ((384, 384, 384), (200, 650, 3000)):
        p = wl.make_problem("N", "T", m, n, k, 1.0, 0.5, seed=7, dist="int", ld_pad=2)
        rc, got = run(p, algo, handle=h)
        assert rc == 0
        assert_bit_exact(p, got)
        check_padding(p, got)


@pytest.mark.parametrize("algo", SPLIT)
def test_promoted_beta_zero_does_not_read_c(handles, algo):
    _, h = handles
    _promoted(h, 64)
    p = wl.make_problem("N", "N", 150, 270, 700, 1.0, 0.0, seed=11)
    p.C[:p.m, :] = np.nan
    rc, got = run(p, algo, handle=h)
    assert rc == 0
    assert not np.isnan(got[:p.m]).any()
    assert_within_bound(p, got, algo=algo)


def test_promotion_lowers_the_error_on_long_k(handles):
    """Log-uniform magnitudes (random sign x 2^U(-20,20)), K = 8192: with
    chunks of 32 the maximum error / bound is lower than without promotion
    for the splits whose products are exact or nearly so."""
    plain, promo = handles
    plain.set_promotion(0)
    _promoted(promo, 32)
    p = wl.split_case(256, 192, 8192, seed=2)
    C64, D = oracle_of(p)
    for algo in ("bf16x6", "bf16x9", "tf32x3"):
        _, a = run(p, algo, handle=plain)
        _, b = run(p, algo, handle=promo)
        ra = oracle.err_report(a[:p.m], C64, D, p.k)["max_ratio"]
        rb = oracle.err_report(b[:p.m], C64, D, p.k)["max_ratio"]
        assert rb < ra, f"{algo}: promoted {rb} not below plain {ra}"


def test_promotion_applies_to_pack_and_compute(handles):
    """The pack-once path takes the handle's setting too: on a shape that
    gb_sgemm does not split along K, pack + compute equals gb_sgemm with the
    same promoted handle bit for bit."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    _, h = handles
    _promoted(h, 64)
    m, n, k = 1100, 1300, 1500
    p = wl.make_problem("N", "N", m, n, k, 1.0, 0.0, seed=12)
    _, want = run(p, "bf16x6", handle=h)
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    C = gb.colmajor(m, n)
    Ap = torch.empty(gb.pack_size("bf16x6", "A", m, k), dtype=torch.uint8, device="cuda")
    Bp = torch.empty(gb.pack_size("bf16x6", "B", n, k), dtype=torch.uint8, device="cuda")
    gb.pack_raw("bf16x6", "A", "N", m, k, A.data_ptr(), p.lda, Ap, handle=h)
    gb.pack_raw("bf16x6", "B", "N", n, k, B.data_ptr(), p.ldb, Bp, handle=h)
    gb.compute_raw("bf16x6", m, n, k, 1.0, Ap, Bp, 0.0, C.data_ptr(), m, handle=h)
    torch.cuda.synchronize()
    assert np.array_equal(gb.to_fortran(C), want[:m])


def test_promoted_bounded_wait_expires_cleanly(handles):
    """A 1 microsecond wait limit makes the promoted kernel's waits run out
    (chunks of 8192: the epilogue waits far longer than that for each): the
    status is reported, and the context still runs a correct GEMM."""
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.Handle()
    h.set_promotion(8192)
    h.set_wait_limit(1)
    p = wl.make_problem("N", "N", 2048, 2048, 16384, 1.0, 0.0, seed=13)
    run(p, "bf16x6", handle=h)
    rc, site = h.device_error()
    assert rc == _lib.GB_ERR_TIMEOUT and site > 0
    h.set_wait_limit(2000000)
    h.set_promotion(32)
    q = wl.make_problem("N", "N", 200, 300, 500, 1.0, 0.0, seed=14)
    rc, got = run(q, "bf16x6", handle=h)
    assert rc == 0
    assert_within_bound(q, got, algo="bf16x6")
    assert h.device_error() == (0, 0)
