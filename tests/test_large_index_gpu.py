"""Outputs past 2^31 elements: M = N = 46400 with ldc = M + 3, so the linear
index i + j*ldc of C crosses 2^31 near column 46279 and every 32-bit index in
an epilogue, a pack or the SIMT kernel would wrap. K = 8 keeps the run short.
Integer data (|a|, |b| <= 2, C in -8..8, beta = 0.5) makes every algorithm
exact, so sampled outputs are compared bit for bit with the oracle run on
the sampled rows and columns as a sub-problem. C (8.6 GB) is filled on the
device with a pattern the host recomputes, and only sampled elements are
read back."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu import torch_gpu

pytestmark = pytest.mark.gpu

M = N = 46400
K = 8
LDC = M + 3
ALPHA, BETA = 1.0, 0.5
ROWS = np.unique(np.r_[0, 1, 127, 128, M // 2, M - 129, M - 2, M - 1,
                       np.random.default_rng(71).integers(0, M, 8)])
COLS = np.unique(np.r_[0, 1, 255, 256, np.arange(46274, 46286), N - 2, N - 1,
                       np.random.default_rng(72).integers(0, N, 8)])


def _c_pattern(i, j):
    """C's initial value at (i, j): an integer in -8..8."""
    return ((7 * i + 13 * j) % 17 - 8).astype(np.float32)


@pytest.fixture(scope="module")
def big_c():
    torch = torch_gpu()
    if torch.cuda.get_device_properties(0).total_memory < 24 * 2 ** 30:
        pytest.skip("needs about 9 GB of device memory for C")
    store = torch.empty((N, LDC), dtype=torch.float32, device="cuda")   # column-major C
    yield store
    del store
    torch.cuda.empty_cache()


def _fill(store):
    import torch
    i = torch.arange(M, device="cuda", dtype=torch.int32)[:, None]
    view = store.t()
    for j0 in range(0, N, 2048):
        j = torch.arange(j0, min(j0 + 2048, N), device="cuda", dtype=torch.int32)[None, :]
        view[:M, j0:j0 + j.shape[1]] = (torch.remainder(7 * i + 13 * j, 17) - 8).float()
    view[M:, :] = float(wl.CANARY)                     # the ldc padding rows


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
@pytest.mark.parametrize("algo", ("simt", "bf16x3", "bf16x6", "tf32x3"))
def test_output_past_2_31_elements(big_c, algo, ta, tb):
    import torch
    import paper_1912_04379_gb300 as gb
    rng = np.random.default_rng(73)
    a_shape = (M, K) if ta == "N" else (K, M)
    b_shape = (K, N) if tb == "N" else (N, K)
    A = np.asfortranarray(rng.integers(-2, 3, a_shape).astype(np.float32))
    B = np.asfortranarray(rng.integers(-2, 3, b_shape).astype(np.float32))
    _, Ad = gb.from_fortran(A)
    _, Bd = gb.from_fortran(B)
    _fill(big_c)
    gb.sgemm_raw(ta, tb, M, N, K, ALPHA, Ad.data_ptr(), a_shape[0], Bd.data_ptr(), b_shape[0],
                 BETA, big_c.data_ptr(), LDC, algo=algo)
    torch.cuda.synchronize()
    ii, jj = np.meshgrid(ROWS, COLS, indexing="ij")
    flat = torch.from_numpy((ii + jj * LDC).ravel().astype(np.int64)).cuda()
    got = torch.take(big_c.reshape(-1), flat).cpu().numpy().reshape(ii.shape)
    # the oracle on the sampled rows of op(A), columns of op(B) and entries of C
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    As = np.asfortranarray(opA[ROWS, :])
    Bs = np.asfortranarray(opB[:, COLS])
    Cs = np.asfortranarray(_c_pattern(ii, jj))
    C64, _ = oracle.sgemm("N", "N", len(ROWS), len(COLS), K, ALPHA, As, len(ROWS), Bs, K,
                          BETA, Cs, len(ROWS))
    assert np.array_equal(got, C64.astype(np.float32))
    # the padding rows of the crossing and the last columns are untouched
    pad_idx = [M + r + j * LDC for j in (46278, 46279, N - 1) for r in range(LDC - M)]
    pad = torch.take(big_c.reshape(-1), torch.tensor(pad_idx, device="cuda")).cpu().numpy()
    assert np.all(pad == np.float32(wl.CANARY))
