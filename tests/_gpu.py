"""Helpers for the GPU parity tests: run one problem through the C ABI and
compare it with the CPU oracle."""
import numpy as np

import oracle
import workloads as wl

ALGOS = ("simt", "tf32x3", "bf16x3", "bf16x6")


def torch_gpu():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run(p, algo, handle=None, check=True):
    """Upload p, run gb_sgemm, return (status, full C storage as Fortran numpy)."""
    import torch
    import paper_1912_04379_gb300 as gb
    _, A = gb.from_fortran(p.A)
    _, B = gb.from_fortran(p.B)
    Cfull, _ = gb.from_fortran(p.C)
    rc = gb.sgemm_raw(p.ta, p.tb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda, B.data_ptr(),
                      p.ldb, p.beta, Cfull.data_ptr(), p.ldc, algo=algo, handle=handle,
                      check=check)
    torch.cuda.synchronize()
    return rc, gb.to_fortran(Cfull)


def oracle_of(p, cols=None):
    return oracle.sgemm(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta,
                        p.C, p.ldc, cols=cols)


def check_padding(p, got):
    """Rows m..ldc-1 of C are padding and must still hold the canary."""
    if p.ldc > p.m:
        assert np.all(got[p.m:, :] == wl.CANARY), "kernel wrote into the padding rows of C"


def assert_within_bound(p, got, cols=None, limit=1.0):
    C64, D = oracle_of(p, cols)
    sub = got[:p.m, :] if cols is None else got[:p.m, cols]
    rep = oracle.err_report(sub, C64, D, p.k)
    assert rep["max_ratio"] <= limit, f"error over bound: {rep}"
    return rep


def assert_bit_exact(p, got):
    C64, _ = oracle_of(p)
    want = C64.astype(np.float32)
    assert np.array_equal(got[:p.m, :], want), \
        f"not bit-exact: {np.count_nonzero(got[:p.m, :] != want)} elements differ"
