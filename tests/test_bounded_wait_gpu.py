"""Bounded waits in the tensor-core kernel: with a wait limit far shorter
than the work, waits expire; the kernel records the site in the device error
word and leaves cleanly (in-flight copies and MMAs drained, TMEM freed), the
host reads GB_ERR_TIMEOUT, and the context stays usable for the next call."""
import numpy as np
import pytest

import workloads as wl
from _gpu import assert_within_bound, run, torch_gpu

pytestmark = pytest.mark.gpu


def test_wait_limit_expiry_is_reported_and_recoverable():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.Handle()
    assert h.device_error() == (0, 0)
    m = n = 2048
    k = 16384
    A = torch.randn(k, m, device="cuda").t()
    B = torch.randn(n, k, device="cuda").t()
    C = torch.empty(n, m, device="cuda").t()
    h.set_wait_limit(1)                      # 1 microsecond: far shorter than one tile's K loop
    gb.sgemm(A, B, C, algo="bf16x3", handle=h)
    rc, site = h.device_error()
    assert rc == _lib.GB_ERR_TIMEOUT and site in (1, 2, 3, 4)
    assert h.device_error() == (0, 0)        # reading clears the word
    h.set_wait_limit(2_000_000)
    p = wl.make_problem("N", "N", 300, 200, 1100, 1.0, 0.5, seed=41)
    rc, got = run(p, "bf16x3", handle=h)
    assert rc == 0
    assert_within_bound(p, got, algo="bf16x3")
    assert h.device_error() == (0, 0)
    with pytest.raises(_lib.GBError):
        h.set_wait_limit(0)


def test_wait_limit_in_the_triangle_and_grouped_kernels():
    """The same bounded waits guard the one-launch SSYRK kernel and the
    grouped kernel: a 1 us limit expires, is reported, and a normal run on
    the same handle afterwards is correct."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    from oracle import blas3
    h = gb.Handle()
    n, k = 1024, 8192
    A = torch.randn(k, n, device="cuda").t().contiguous().t()      # column-major n x k
    C = gb.colmajor(n, n, fill=0.0)
    h.set_wait_limit(1)
    gb.ssyrk_raw("L", "N", n, k, 1.0, A.data_ptr(), n, 0.0, C.data_ptr(), n, algo="bf16x3",
                 handle=h)
    rc, site = h.device_error()
    assert rc == _lib.GB_ERR_TIMEOUT and site in (1, 2, 3, 4)
    probs = [wl.make_problem("N", "T", 300, 280, 4000, 1.0, 0.0, seed=90 + i) for i in range(8)]
    buf, tuples, views = gb.upload_problems(probs)
    plan = gb.GroupedPlan(tuples, algo="bf16x6", handle=h)
    plan.run()
    rc, site = h.device_error()
    assert rc == _lib.GB_ERR_TIMEOUT and site in (1, 2, 3, 4)
    plan.close()
    # recovery: normal limit, correct results on the same handle
    h.set_wait_limit(2_000_000)
    rng = np.random.default_rng(91)
    Ah = np.asfortranarray(rng.uniform(-1, 1, (300, 700)).astype(np.float32))
    Ch = np.asfortranarray(np.zeros((300, 300), dtype=np.float32))
    Ad, _ = gb.from_fortran(Ah)
    Cd, _ = gb.from_fortran(Ch)
    gb.ssyrk_raw("U", "N", 300, 700, 1.0, Ad.data_ptr(), 300, 0.0, Cd.data_ptr(), 300,
                 algo="bf16x3", handle=h)
    torch.cuda.synchronize()
    assert h.device_error() == (0, 0)
    C64, D = blas3.ssyrk("U", "N", 300, 700, 1.0, Ah, 300, 0.0, Ch, 300)
    got = gb.to_fortran(Cd)
    iu = np.triu_indices(300)
    from _gpu import split_extra
    bound = (2 * 700 * 2.0 ** -24 + split_extra("bf16x3", 700)) * D[iu]
    assert np.all(np.abs(got[iu] - C64[iu]) <= bound)
