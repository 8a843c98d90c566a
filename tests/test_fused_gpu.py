"""The split fused into the tensor-core kernel (TMA reads FP32 operands, converter
warps split them in shared memory) against the two-pass path (split/pack pass,
then the kernel), and both against the FP64 oracle.

The fused kernel consumes K in 32-element stages, like the two-pass kernel's
64-byte-row variant, which the two-pass path uses when K > 2048: there the two
paths form the same terms and issue the same MMAs in the same order, so their
results must be bit-identical. For K <= 2048 the two-pass path uses 64-element
stages (a different accumulation order), so only the error bound applies."""
import numpy as np
import pytest

import workloads as wl
from _gpu import aligned_problem as _aligned_problem
from _gpu import assert_bit_exact, assert_within_bound, check_padding, torch_gpu

pytestmark = pytest.mark.gpu
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


def _run_both(p, algo):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    fused, twopass = gb.Handle(), gb.Handle()
    fused.set_fused_split(True)
    twopass.set_fused_split(False)
    for h in (fused, twopass):          # the skinny-product kernel would take (64, 2048, 4096)
        h.set_skinny_split(False)
    outs = []
    for h in (fused, twopass):
        _, A = gb.from_fortran(p.A)
        _, B = gb.from_fortran(p.B)
        Cfull, _ = gb.from_fortran(p.C)
        assert A.data_ptr() % 16 == 0 and B.data_ptr() % 16 == 0
        gb.sgemm_raw(p.ta, p.tb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda, B.data_ptr(),
                     p.ldb, p.beta, Cfull.data_ptr(), p.ldc, algo=algo, handle=h)
        torch.cuda.synchronize()
        outs.append(gb.to_fortran(Cfull))
        assert h.device_error() == (0, 0)
    return outs


SHAPES = [(8, 8, 8), (128, 256, 64), (129, 257, 33), (300, 260, 1000), (256, 512, 2500),
          (1000, 700, 3000), (64, 2048, 4096), (300, 270, 2100)]


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6"))
def test_fused_equals_two_pass(algo, shape, ta, tb):
    m, n, k = shape
    p = _aligned_problem(ta, tb, m, n, k, 1.25, -0.5, seed=m + 3 * n + 7 * k)
    fused, twopass = _run_both(p, algo)
    if k > 2048 or k <= 16:
        assert np.array_equal(fused, twopass), \
            f"{np.count_nonzero(fused != twopass)} elements differ between fused and two-pass"
    assert_within_bound(p, fused, algo=algo)
    assert_within_bound(p, twopass, algo=algo)
    check_padding(p, fused)


@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6"))
def test_fused_integer_bit_exact(algo):
    p = _aligned_problem("T", "N", 260, 300, 2100, 1.0, 0.5, seed=71, dist="int")   # K > 2048
    fused, twopass = _run_both(p, algo)
    assert_bit_exact(p, fused)
    assert np.array_equal(fused, twopass)


@pytest.mark.parametrize("ta,tb", TRANS)
def test_fused_log_uniform_magnitudes(ta, tb):
    p = _aligned_problem(ta, tb, 200, 330, 2200, 1.0, 0.0, seed=72, dist="logu")
    fused, twopass = _run_both(p, "bf16x3")
    assert np.array_equal(fused, twopass)
    assert_within_bound(p, fused, algo="bf16x3")


def test_fused_special_values_match_two_pass():
    """Non-finite and near-overflow inputs take the exact scalar split in both paths."""
    p = _aligned_problem("N", "N", 64, 64, 2080, 1.0, 0.0, seed=73)
    p.A[3, 5] = np.inf
    p.A[7, 9] = -np.inf
    p.B[2, 11] = np.nan
    p.A[10, 10] = np.float32(3.4e38)
    p.B[10, 20] = np.float32(-3.39e38)
    fused, twopass = _run_both(p, "bf16x6")
    same = (fused == twopass) | (np.isnan(fused) & np.isnan(twopass))
    assert np.all(same)
