"""Pack-once / compute-many: gb_sgemm_pack + gb_sgemm_compute must give the
same bits as gb_sgemm when gb_sgemm does not split K (same kernels, same
order), and a packed operand can be reused across calls."""
import numpy as np
import pytest

import workloads as wl
from _gpu import assert_within_bound, torch_gpu

pytestmark = pytest.mark.gpu
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("algo", ("tf32x3", "bf16x3", "bf16x6"))
def test_pack_compute_equals_sgemm(algo, ta, tb):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    # K < 1024: gb_sgemm does not split K here, so both paths run the same
    # kernels in the same order
    p = wl.make_problem(ta, tb, 300, 260, 1000, 0.5, -1.5, seed=31, ld_pad=5)
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    C1full, _ = gb.from_fortran(p.C)
    C2full, _ = gb.from_fortran(p.C)
    gb.sgemm_raw(ta, tb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda, B.data_ptr(), p.ldb,
                 p.beta, C1full.data_ptr(), p.ldc, algo=algo)
    Ap = torch.empty(gb.pack_size(algo, "A", p.m, p.k), dtype=torch.uint8, device="cuda")
    Bp = torch.empty(gb.pack_size(algo, "B", p.n, p.k), dtype=torch.uint8, device="cuda")
    gb.pack_raw(algo, "A", ta, p.m, p.k, A.data_ptr(), p.lda, Ap)
    gb.pack_raw(algo, "B", tb, p.n, p.k, B.data_ptr(), p.ldb, Bp)
    gb.compute_raw(algo, p.m, p.n, p.k, p.alpha, Ap, Bp, p.beta, C2full.data_ptr(), p.ldc)
    torch.cuda.synchronize()
    c1, c2 = gb.to_fortran(C1full), gb.to_fortran(C2full)
    assert np.array_equal(c1, c2)
    assert_within_bound(p, c2, algo=algo)


def test_packed_operand_reuse():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    algo = "bf16x6"
    p1 = wl.make_problem("N", "N", 200, 150, 300, 1.0, 0.0, seed=32)
    p2 = wl.make_problem("N", "N", 200, 150, 300, 1.0, 0.0, seed=33)
    p2.B = p1.B                                        # same B, different A
    Bp = torch.empty(gb.pack_size(algo, "B", 150, 300), dtype=torch.uint8, device="cuda")
    _, B = gb.from_fortran(p1.B)
    gb.pack_raw(algo, "B", "N", 150, 300, B.data_ptr(), 300, Bp)
    for p in (p1, p2):
        _, A = gb.from_fortran(p.A)
        Ap = torch.empty(gb.pack_size(algo, "A", 200, 300), dtype=torch.uint8, device="cuda")
        gb.pack_raw(algo, "A", "N", 200, 300, A.data_ptr(), 200, Ap)
        Cfull, _ = gb.from_fortran(p.C)
        gb.compute_raw(algo, 200, 150, 300, 1.0, Ap, Bp, 0.0, Cfull.data_ptr(), 200)
        torch.cuda.synchronize()
        assert_within_bound(p, gb.to_fortran(Cfull), algo=algo)


def test_pack_argument_errors():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    X = torch.zeros(64, 64, device="cuda")
    buf = torch.empty(gb.pack_size("bf16x3", "A", 64, 64), dtype=torch.uint8, device="cuda")
    assert gb.pack_raw("bf16x3", "Z", "N", 64, 64, X.data_ptr(), 64, buf, check=False) == -1
    assert gb.pack_raw("bf16x3", "A", "N", 64, 64, X.data_ptr(), 63, buf, check=False) == -8
    assert gb.pack_raw("bf16x3", "A", "N", 64, 64, X.data_ptr(), 64, buf[:100],
                       check=False) == _lib.GB_ERR_WORKSPACE
    assert gb.pack_raw("simt", "A", "N", 64, 64, X.data_ptr(), 64, buf,
                       check=False) == _lib.GB_ERR_UNSUPPORTED
