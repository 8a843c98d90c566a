"""The GPU error report (the library's only FP64 kernel) against the CPU
definition in oracle.err_report: same ratios bit for bit, so the maximum and
the lower median agree exactly; the sums agree to rounding."""
import numpy as np
import pytest

import oracle
from _gpu import torch_gpu

pytestmark = pytest.mark.gpu


def _cm(t2d_numpy_f, torch, dtype):
    # Fortran numpy (m, n) -> column-major CUDA tensor view (m, n)
    return torch.from_numpy(np.ascontiguousarray(t2d_numpy_f.T)).to("cuda", dtype).t()


def _compare(C, C64, D, k):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    got = gb.err_report(_cm(C, torch, torch.float32), _cm(C64, torch, torch.float64),
                        _cm(D, torch, torch.float64), k)
    want = oracle.err_report(C, C64, D, k)
    assert got["max_ratio"] == want["max_ratio"]
    assert got["median_ratio"] == want["median_ratio"]
    assert got["n_fail"] == want["n_fail"] and got["count"] == want["count"]
    if np.isfinite(want["normwise"]):
        assert got["normwise"] == pytest.approx(want["normwise"], rel=1e-10, abs=1e-300)
    return got


@pytest.mark.parametrize("shape", [(1, 1), (7, 3), (300, 200), (1024, 999)])
def test_err_report_matches_definition(shape):
    m, n = shape
    rng = np.random.default_rng(m * n)
    C64 = np.asfortranarray(rng.normal(size=(m, n)))
    D = np.asfortranarray(np.abs(C64) + rng.uniform(0.5, 2.0, size=(m, n)))
    k = 100
    bound = oracle.bound(D, k)
    C = np.asfortranarray((C64 + rng.uniform(-2, 2, size=(m, n)) * bound).astype(np.float32))
    _compare(C, C64, D, k)


def test_err_report_special_values():
    m, n = 64, 40
    rng = np.random.default_rng(5)
    C64 = np.asfortranarray(rng.normal(size=(m, n)))
    D = np.asfortranarray(np.abs(C64) + 1.0)
    C = np.asfortranarray(C64.astype(np.float32))
    D[0, 0] = 0.0; C64[0, 0] = 0.0; C[0, 0] = 0.0               # zero bound, exact: ratio 0
    D[1, 0] = 0.0; C64[1, 0] = 0.0; C[1, 0] = 1e-30             # zero bound, nonzero error: inf
    C64[2, 0] = np.nan; C[2, 0] = np.nan                        # both NaN: agree
    C64[3, 0] = np.inf; C[3, 0] = np.inf                        # same infinity: agree
    C64[4, 0] = 1.0; C[4, 0] = np.nan                           # one side NaN: inf
    C64[5, 0] = -np.inf; C[5, 0] = np.inf                       # opposite infinities: inf
    got = _compare(C, C64, D, 3)
    assert got["max_ratio"] == np.inf and got["n_fail"] == 3


def test_err_report_k_zero_and_large_count():
    m, n = 4096, 1500                                           # 6.1M keys: many blocks
    rng = np.random.default_rng(9)
    C64 = np.asfortranarray(rng.normal(size=(m, n)))
    D = np.asfortranarray(np.abs(C64) + 0.25)
    C = np.asfortranarray(C64.astype(np.float32))
    _compare(C, C64, D, 0)
