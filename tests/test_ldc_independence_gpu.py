"""Results do not depend on C's leading dimension: the same problem stored at
an ldc that is a multiple of 4 (16-byte aligned columns) and at one that is
not gives bit-identical C, the padding rows (ldc > M) keep their canary, and
both are within the oracle's bound. (This also guards any epilogue variant
chosen by the alignment of C.)"""
import numpy as np
import pytest

import workloads as wl
from _gpu import assert_within_bound, check_padding, run, torch_gpu

pytestmark = pytest.mark.gpu
SHAPES = [(300, 260, 100), (128, 256, 64), (129, 257, 33), (1000, 700, 3000), (64, 4100, 256),
          (4096, 4096, 64)]


def _with_ldc(p, ldc):
    """The same problem with C stored at leading dimension ldc (canary padding)."""
    C = np.full((ldc, max(p.n, 1)), wl.CANARY, dtype=np.float32, order="F")
    C[:p.m, :p.n] = p.C[:p.m, :p.n]
    return wl.Problem(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.beta, p.A, p.lda, p.B, p.ldb, C, ldc)


@pytest.mark.parametrize("beta", (0.0, 0.5))
@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6", "tf32x3"))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_results_independent_of_ldc(shape, algo, beta):
    torch_gpu()
    m, n, k = shape
    p = wl.make_problem("N", "T", m, n, k, 1.5, beta, seed=m + n + k)
    ld_tma = (m + 3) // 4 * 4 + 4               # a multiple of 4
    ld_plain = ld_tma + 1                       # not a multiple of 4
    outs = []
    for ldc in (ld_tma, ld_plain):
        q = _with_ldc(p, ldc)
        rc, got = run(q, algo)
        assert rc == 0
        check_padding(q, got)
        assert_within_bound(q, got, algo=algo)
        outs.append(got[:m, :n])
    assert np.array_equal(outs[0], outs[1])
