"""Non-finite and near-overflow inputs, against the oracle's IEEE FP64 result.

SIMT forms each product in FP32 with IEEE semantics, so its NaN and +-Inf
positions equal the oracle's. The split algorithms split a non-finite value
a as (a, 0[, 0]); a product of an infinite term with a zero term of the other
operand is NaN, so an infinite result can come out as NaN. What holds for
them: the non-finite positions equal the oracle's, and every finite
element is within the algorithm's bound. Finite values near the FP32 limit
must not overflow in the split (a leading term that would round to infinity
is truncated instead)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu import run, split_extra, torch_gpu

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _problem(ta, tb, seed):
    p = wl.make_problem(ta, tb, 70, 50, 40, 1.0, 0.5, seed=seed, ld_pad=1)
    # op(A)[3, 5] = +inf, op(A)[10, 7] = -inf, op(B)[5, 20] = nan
    def set_op(X, trans, i, j, v):
        if trans == "N":
            X[i, j] = v
        else:
            X[j, i] = v
    set_op(p.A, ta, 3, 5, np.inf)
    set_op(p.A, ta, 10, 7, -np.inf)
    set_op(p.B, tb, 5, 20, np.nan)
    return p


@pytest.mark.parametrize("algo", ("simt", "tf32x3", "bf16x3", "bf16x6", "bf16x9", "fp16x3"))
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_nonfinite_positions(algo, ta, tb):
    torch_gpu()
    p = _problem(ta, tb, seed=11)
    rc, got = run(p, algo)
    assert rc == 0
    C64, D = oracle.sgemm(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta,
                          p.C, p.ldc)
    g = got[:p.m, :].astype(np.float64)
    bad64 = ~np.isfinite(C64)
    assert bad64.any()
    assert np.array_equal(~np.isfinite(g), bad64)
    if algo == "simt":
        assert np.array_equal(np.isnan(g), np.isnan(C64))
        inf = np.isinf(C64)
        assert np.array_equal(g[inf], C64[inf])
    fin = ~bad64
    bound = (2 * p.k * U + split_extra(algo, p.k)) * D[fin]
    assert np.all(np.abs(g[fin] - C64[fin]) <= bound)


@pytest.mark.parametrize("algo", ("simt", "tf32x3", "bf16x3", "bf16x6", "bf16x9", "fp16x3"))
def test_near_overflow_stays_finite(algo):
    torch_gpu()
    rng = np.random.default_rng(12)
    p = wl.make_problem("N", "N", 40, 30, 8, 1.0, 0.0, seed=12)
    p.A[:40, :8] = rng.choice([-1.0, 1.0], (40, 8)) * rng.uniform(3.0e38, 3.4e38, (40, 8))
    p.B[:8, :30] = 0.0
    p.B[rng.integers(0, 8, 30), np.arange(30)] = rng.uniform(0.5, 1.0, 30)   # one nonzero per column
    p.A = np.asfortranarray(p.A.astype(np.float32))
    p.B = np.asfortranarray(p.B.astype(np.float32))
    rc, got = run(p, algo)
    C64, D = oracle.sgemm(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta,
                          p.C, p.ldc)
    g = got[:p.m, :].astype(np.float64)
    assert np.all(np.isfinite(C64)) and np.all(np.isfinite(g))
    bound = (2 * p.k * U + split_extra(algo, p.k)) * D
    assert np.all(np.abs(g - C64) <= bound)
