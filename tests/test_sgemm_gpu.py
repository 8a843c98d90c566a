"""GPU parity: every algorithm against the FP64 CPU oracle, through the C ABI.

Acceptance per element: |C - C64| <= 2 * max(K,1) * 2^-24 * D (D = |alpha||op(A)||op(B)|
+ |beta||C|), and bit-exact equality on integer-valued inputs whose partial sums stay
below 2^24. Padding rows of C (ld > M) must keep their canary value.
"""
import numpy as np
import pytest

import workloads as wl
from _gpu import ALGOS, assert_bit_exact, assert_within_bound, check_padding, run, torch_gpu

pytestmark = pytest.mark.gpu
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]
SPLIT = ("tf32x3", "bf16x3", "bf16x6", "bf16x9", "fp16x3")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch_gpu()


# --------------------------------------------------------------- 384^3 ----

@pytest.mark.parametrize("algo", ALGOS)
def test_plain_384(algo):
    p = wl.plain_384()
    rc, got = run(p, algo)
    assert rc == 0
    assert_within_bound(p, got, algo=algo)


@pytest.mark.parametrize("algo", ALGOS)
def test_plain_384_integer_bit_exact(algo):
    p = wl.plain_384(integer=True)
    rc, got = run(p, algo)
    assert_bit_exact(p, got)


# ------------------------------------------------- padded-stride sweep ----

@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("n", (16, 100, 257, 512, 1000, 1023))
def test_simt_sweep(n, ta, tb):
    p = wl.sweep_case(n, ta, tb)
    rc, got = run(p, "simt")
    assert_within_bound(p, got)
    check_padding(p, got)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("n", (2048, 4096, 8192))
def test_simt_sweep_large_sampled(n, ta, tb):
    p = wl.sweep_case(n, ta, tb)
    rc, got = run(p, "simt")
    cols = np.unique(np.r_[0, 1, n // 2, n - 1, np.random.default_rng(n).integers(0, n, 4)])
    assert_within_bound(p, got, cols=cols)
    check_padding(p, got)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("algo", SPLIT)
@pytest.mark.parametrize("n", (100, 257, 1000))
def test_split_sweep(algo, n, ta, tb):
    p = wl.sweep_case(n, ta, tb)
    rc, got = run(p, algo)
    assert_within_bound(p, got, algo=algo)
    check_padding(p, got)


# ----------------------------------------------------- ragged shapes ----

RAGGED = [(1, 1, 1), (7, 5, 3), (33, 17, 65), (127, 129, 31), (129, 255, 257),
          (300, 520, 100), (1, 300, 7), (300, 1, 77), (128, 256, 64), (257, 513, 129)]


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("shape", RAGGED, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("algo", ALGOS)
def test_ragged(algo, shape, ta, tb):
    m, n, k = shape
    p = wl.make_problem(ta, tb, m, n, k, -0.75, 1.25, seed=m * 7919 + n * 31 + k, ld_pad=3)
    rc, got = run(p, algo)
    assert rc == 0
    assert_within_bound(p, got, algo=algo)
    check_padding(p, got)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("algo", ALGOS)
def test_ragged_integer_bit_exact(algo, ta, tb):
    p = wl.make_problem(ta, tb, 257, 130, 1029, 1.0, 0.5, seed=21, dist="int", ld_pad=5)
    rc, got = run(p, algo)
    assert_bit_exact(p, got)
    check_padding(p, got)


def test_persistent_many_tiles():
    """More output tiles than SMs: every CTA walks several tiles and both TMEM
    accumulators are reused."""
    for algo in SPLIT:
        p = wl.make_problem("N", "N", 4100, 4100, 64, 1.0, -1.0, seed=22)
        rc, got = run(p, algo)
        cols = np.r_[0:3, 255:258, 4097:4100]
        assert_within_bound(p, got, cols=cols, algo=algo)


# ------------------------------------------------ log-uniform magnitudes --

@pytest.mark.parametrize("k", (8, 64, 1000))
@pytest.mark.parametrize("algo", ("simt", "tf32x3", "bf16x6", "bf16x9", "fp16x3"))
def test_log_uniform_small(algo, k):
    p = wl.make_problem("N", "N", 200, 150, k, 1.0, 0.0, seed=23, dist="logu")
    rc, got = run(p, algo)
    assert_within_bound(p, got, algo=algo)


def test_bf16x3_log_uniform_large_k():
    p = wl.make_problem("T", "N", 200, 150, 4096, 1.0, 0.0, seed=24, dist="logu")
    rc, got = run(p, "bf16x3")
    assert_within_bound(p, got, algo="bf16x3")


# ------------------------------------------------ BLAS special cases ----

@pytest.mark.parametrize("algo", ALGOS)
def test_quick_return_and_alpha_zero(algo):
    import paper_1912_04379_gb300 as gb
    torch = torch_gpu()
    m, n, k = 37, 29, 11
    A = torch.full((k, m), float("nan"), device="cuda").t()       # column-major m x k
    B = torch.full((n, k), float("nan"), device="cuda").t()
    C0 = torch.randn(n, m, device="cuda").t()
    # alpha = 0, beta = 1: nothing happens (and NaN A/B are never read)
    C = C0.clone()
    gb.sgemm(A, B, C, alpha=0.0, beta=1.0, algo=algo)
    torch.cuda.synchronize()
    assert torch.equal(C, C0)
    # alpha = 0, beta = -2: C = beta*C, A and B not read
    C = C0.clone()
    gb.sgemm(A, B, C, alpha=0.0, beta=-2.0, algo=algo)
    torch.cuda.synchronize()
    assert torch.equal(C, -2.0 * C0)
    # beta = 0: C not read (NaN in C must not propagate)
    A2 = torch.randn(k, m, device="cuda").t()
    B2 = torch.randn(n, k, device="cuda").t()
    C = torch.full((n, m), float("nan"), device="cuda").t()
    gb.sgemm(A2, B2, C, alpha=1.0, beta=0.0, algo=algo)
    torch.cuda.synchronize()
    assert torch.isfinite(C).all()
    # K = 0: C = beta*C
    Ak = torch.empty(0, m, device="cuda").t()
    Bk = torch.empty(n, 0, device="cuda").t()
    C = C0.clone()
    gb.sgemm(Ak, Bk, C, alpha=1.0, beta=0.5, algo=algo)
    torch.cuda.synchronize()
    assert torch.equal(C, 0.5 * C0)
    # M = 0 / N = 0: nothing enqueued
    gb.sgemm(A2[:0], B2, C[:0], alpha=1.0, beta=0.0, algo=algo)
    gb.sgemm(A2, B2[:, :0], C[:, :0], alpha=1.0, beta=0.0, algo=algo)


def test_workspace_errors():
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    torch = torch_gpu()
    A = torch.randn(64, 64, device="cuda")
    need = gb.workspace_size("bf16x3", "N", "N", 64, 64, 64)
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    small = ws[: need - 1]
    C = torch.empty_like(A)
    rc = gb.sgemm_raw("N", "N", 64, 64, 64, 1.0, A.data_ptr(), 64, A.data_ptr(), 64, 0.0,
                      C.data_ptr(), 64, algo="bf16x3", workspace=small, check=False)
    assert rc == _lib.GB_ERR_WORKSPACE
    mis = ws[8: 8 + need]
    rc = gb.sgemm_raw("N", "N", 64, 64, 64, 1.0, A.data_ptr(), 64, A.data_ptr(), 64, 0.0,
                      C.data_ptr(), 64, algo="bf16x3", workspace=mis, check=False)
    assert rc == _lib.GB_ERR_WORKSPACE
    rc = gb.sgemm_raw("N", "N", 64, 64, 64, 1.0, A.data_ptr(), 64, A.data_ptr(), 64, 0.0,
                      C.data_ptr(), 64, algo="bf16x3", workspace=ws[:need], check=False)
    assert rc == 0
    torch.cuda.synchronize()


def test_device_error_word_clean():
    import paper_1912_04379_gb300 as gb
    torch_gpu()
    h = gb.default_handle()
    p = wl.make_problem("N", "N", 300, 300, 300, 1.0, 0.0, seed=25)
    for algo in SPLIT:
        rc, got = run(p, algo, handle=h)
        assert h.device_error() == (0, 0)


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("algo", SPLIT)
def test_long_k_ragged(algo, ta, tb):
    """K > 2048 selects the four-stage, 64-byte-row pipeline; ragged M, N, K."""
    p = wl.make_problem(ta, tb, 300, 270, 2500, 1.0, -0.5, seed=26, ld_pad=3)
    rc, got = run(p, algo)
    assert_within_bound(p, got, algo=algo)
    check_padding(p, got)


@pytest.mark.parametrize("algo", SPLIT)
def test_long_k_integer_bit_exact(algo):
    p = wl.make_problem("T", "N", 140, 260, 4100, 1.0, 0.5, seed=27, dist="int", ld_pad=1)
    rc, got = run(p, algo)
    assert_bit_exact(p, got)


# ------------------------------------------------------------- split-K ----

@pytest.mark.parametrize("algo", SPLIT)
def test_split_k_small_full_check(algo):
    """Few output tiles and a long K: the K range is cut into slices whose
    partial sums are reduced in a fixed order (beta != 0 goes through the reduce)."""
    p = wl.make_problem("N", "T", 200, 300, 3000, 0.5, 0.5, seed=28, ld_pad=2)
    rc, got = run(p, algo)
    assert_within_bound(p, got, algo=algo)
    check_padding(p, got)


@pytest.mark.parametrize("algo", SPLIT)
def test_split_k_integer_bit_exact(algo):
    p = wl.make_problem("T", "T", 100, 100, 5000, 1.0, 0.5, seed=29, dist="int", ld_pad=1)
    rc, got = run(p, algo)
    assert_bit_exact(p, got)


def test_split_k_factor_is_used_in_workspace():
    import paper_1912_04379_gb300 as gb
    base = 2 * 2 * 8192 * (64 + 8192)             # packed A + B, BF16 x 2 terms, K = 8192
    ws = gb.workspace_size("bf16x3", "N", "N", 64, 8192, 8192)
    assert ws == base + 4 * 64 * 8192 * 4         # 4 slices of FP32 partials
    assert gb.workspace_size("bf16x3", "N", "N", 8192, 8192, 8192) == 2 * 2 * 8192 * 16384


# ----------------------------------------- full-size split shapes (sampled) --

_SPLIT_CACHE = {}


def _split_problem(shape):
    if shape not in _SPLIT_CACHE:
        _SPLIT_CACHE.clear()
        _SPLIT_CACHE[shape] = wl.split_case(*shape)
    return _SPLIT_CACHE[shape]


@pytest.mark.parametrize("algo", SPLIT)
@pytest.mark.parametrize("shape", wl.SPLIT_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_split_shapes_full_size_sampled(shape, algo):
    p = _split_problem(shape)
    rc, got = run(p, algo)
    assert rc == 0
    n = p.n
    cols = np.unique(np.r_[0, n - 1, np.random.default_rng(n + p.k).integers(0, n, 6)])
    assert_within_bound(p, got, cols=cols, algo=algo)


# ------------------------------------------------- all nine products ----

@pytest.mark.parametrize("k", (1, 2, 3, 5))
@pytest.mark.parametrize("ta,tb", TRANS)
def test_bf16x9_tiny_k(k, ta, tb):
    """All nine products: every a*b is formed exactly, so only the tensor
    core's FP32 accumulation (not round-to-nearest) adds to the plain bound."""
    p = wl.make_problem(ta, tb, 150, 140, k, 1.0, -0.75, seed=40 + k, dist="logu", ld_pad=2)
    rc, got = run(p, "bf16x9")
    assert_within_bound(p, got, algo="bf16x9")
    check_padding(p, got)


def test_bf16x9_split_k():
    """BF16X9 on a split-K shape (64 x 2000 x 6000, beta != 0): plain bound."""
    p = wl.make_problem("N", "T", 64, 2000, 6000, 0.5, 0.5, seed=45, ld_pad=1)
    rc, got = run(p, "bf16x9")
    cols = np.unique(np.r_[0, 1, 999, 1999, np.random.default_rng(45).integers(0, 2000, 8)])
    assert_within_bound(p, got, cols=cols)
    check_padding(p, got)


# ------------------------------------------------- tile-count independence --

@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6"))
def test_result_does_not_depend_on_the_tile_count(algo):
    """Each output element accumulates the same K sequence whatever the number
    of tiles (and so whatever tiles land in the persistent grid's last
    round): two problems that differ only in N agree bit for bit on their
    common columns."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, k = 4096, 512
    bn = 256 if algo == "bf16x3" else 128
    n_wide = 20 * bn                              # 32 x 20 tiles of 128 x 256 (or 40 x 128)
    n_narrow = 19 * bn
    g = torch.Generator(device="cuda").manual_seed(42)
    A = (torch.rand((k, m), device="cuda", generator=g) * 2 - 1).t()
    B = (torch.rand((n_wide, k), device="cuda", generator=g) * 2 - 1).t()
    outs = []
    for n in (n_wide, n_narrow):
        C = gb.colmajor(m, n)
        gb.sgemm(A, B[:, :n], C, algo=algo)
        torch.cuda.synchronize()
        outs.append(C)
    assert torch.equal(outs[0][:, :n_narrow], outs[1])
    # and the wide result (tail units included) is within the bound
    p = wl.Problem("N", "N", m, n_wide, k, 1.0, 0.0,
                   np.asfortranarray(A.cpu().numpy()), m,
                   np.asfortranarray(B.cpu().numpy()), k,
                   np.zeros((m, n_wide), dtype=np.float32, order="F"), m)
    got = np.asfortranarray(outs[0].cpu().numpy())
    cols = np.r_[n_wide - bn:n_wide:7, 0:3]
    assert_within_bound(p, got, cols=cols, algo=algo)
