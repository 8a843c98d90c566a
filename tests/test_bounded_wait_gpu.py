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
