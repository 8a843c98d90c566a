"""GPU parity of gb_ssyrk and gb_strsm against the FP64 oracle (oracle/blas3.py).

SSYRK: every element of the `uplo` triangle within the SGEMM bound
(2 max(K,1) u + e_algo) D of the algorithm that ran (the one-launch
tensor-core triangle for a split algorithm; GEMM recursion with FP32
diagonal blocks for SIMT); the other triangle holds NaN and must come back
untouched; padding rows keep their canary; integer data is bit-exact.

STRSM: the solution is checked through its residual, a property that holds
at any size: with s = m (side 'L') or n (side 'R') and the recursion depth d,
  |op(A) X - alpha B| <= ((2s + 2) u + d e_algo) |op(A)||X| + 2u |alpha B|
elementwise (backward stability of substitution plus one GEMM bound per
recursion level); integer unit-triangular systems are solved exactly; and
for well-conditioned A the solution tracks the oracle's X.
"""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import blas3
from _gpu import auto_algo, split_extra, torch_gpu

pytestmark = pytest.mark.gpu
U = 2.0 ** -24
COMBOS = list(itertools.product("LR", "LU", "NT", "NU"))


def _resolve(algo, k):
    if algo != "auto":
        return algo
    return auto_algo(k)


def _dev(arr):
    import paper_1912_04379_gb300 as gb
    store, _ = gb.from_fortran(np.asfortranarray(arr, dtype=np.float32))
    return store


# ------------------------------------------------------------------ SSYRK --

def _syrk_case(uplo, trans, n, k, alpha, beta, seed, dist="uniform", pad=3):
    rng = np.random.default_rng(seed)
    gen = {"uniform": wl.uniform, "int": wl.int_uniform, "logu": wl.log_uniform_signed}[dist]
    ar, ac = (n, k) if trans == "N" else (k, n)
    A = gen(rng, ar, ac, max(ar, 1) + pad)
    C = gen(rng, n, n, max(n, 1) + pad, pad=wl.CANARY)
    i, j = np.indices((n, n))
    other = (i < j) if uplo == "L" else (i > j)
    Cv = C[:n, :n]
    Cv[other] = np.nan
    return A, C


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
@pytest.mark.parametrize("n,k", [(1, 1), (100, 50), (129, 7), (300, 200), (520, 1100)])
@pytest.mark.parametrize("algo", ("simt", "bf16x6", "auto"))
def test_ssyrk_against_oracle(algo, n, k, uplo, trans):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    alpha, beta = 1.25, -0.5
    A, C = _syrk_case(uplo, trans, n, k, alpha, beta, seed=n + k)
    Ad, Cd = _dev(A), _dev(C)
    gb.ssyrk_raw(uplo, trans, n, k, alpha, Ad.data_ptr(), A.shape[0], beta, Cd.data_ptr(),
                 C.shape[0], algo=algo)
    torch.cuda.synchronize()
    got = gb.to_fortran(Cd)
    C64, D = blas3.ssyrk(uplo, trans, n, k, alpha, A, A.shape[0], beta, C, C.shape[0])
    mask = ~np.isnan(C64)
    bound = (2 * max(k, 1) * U + split_extra(_resolve(algo, k), k)) * D
    err = np.abs(got[:n, :n] - C64)
    assert np.all(err[mask] <= bound[mask]), float(np.max(err[mask] / bound[mask]))
    assert np.all(np.isnan(got[:n, :n][~mask]))            # other triangle untouched
    assert np.all(got[n:, :] == wl.CANARY)                 # padding rows


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
@pytest.mark.parametrize("n,k", [(300, 20), (520, 2100)])
@pytest.mark.parametrize("algo", ("tf32x3", "bf16x3", "bf16x9"))
def test_ssyrk_tensor_core_algorithms(algo, n, k, uplo, trans):
    """The one-launch triangle kernel for every split (both stage widths)."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    A, C = _syrk_case(uplo, trans, n, k, -0.75, 1.5, seed=3 * n + k, dist="logu")
    Ad, Cd = _dev(A), _dev(C)
    gb.ssyrk_raw(uplo, trans, n, k, -0.75, Ad.data_ptr(), A.shape[0], 1.5, Cd.data_ptr(),
                 C.shape[0], algo=algo)
    torch.cuda.synchronize()
    assert gb.default_handle().device_error() == (0, 0)
    got = gb.to_fortran(Cd)
    C64, D = blas3.ssyrk(uplo, trans, n, k, -0.75, A, A.shape[0], 1.5, C, C.shape[0])
    mask = ~np.isnan(C64)
    bound = (2 * max(k, 1) * U + split_extra(algo, k)) * D
    err = np.abs(got[:n, :n] - C64)
    assert np.all(err[mask] <= bound[mask]), float(np.max(err[mask] / bound[mask]))
    assert np.all(np.isnan(got[:n, :n][~mask]))
    assert np.all(got[n:, :] == wl.CANARY)


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_ssyrk_integer_bit_exact(uplo, trans):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    n, k = 333, 1500
    A, C = _syrk_case(uplo, trans, n, k, 1.0, 0.5, seed=5, dist="int")
    Ad, Cd = _dev(A), _dev(C)
    gb.ssyrk_raw(uplo, trans, n, k, 1.0, Ad.data_ptr(), A.shape[0], 0.5, Cd.data_ptr(),
                 C.shape[0], algo="auto")
    torch.cuda.synchronize()
    got = gb.to_fortran(Cd)[:n, :n]
    C64, _ = blas3.ssyrk(uplo, trans, n, k, 1.0, A, A.shape[0], 0.5, C, C.shape[0])
    mask = ~np.isnan(C64)
    assert np.array_equal(got[mask], C64[mask].astype(np.float32))


def test_ssyrk_special_cases():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    n, k = 200, 30
    # beta = 0: C (NaN) is not read
    A, C = _syrk_case("L", "N", n, k, 1.0, 0.0, seed=6)
    C[:n, :n] = np.nan
    Ad, Cd = _dev(A), _dev(C)
    gb.ssyrk_raw("L", "N", n, k, 1.0, Ad.data_ptr(), A.shape[0], 0.0, Cd.data_ptr(), C.shape[0])
    torch.cuda.synchronize()
    got = gb.to_fortran(Cd)[:n, :n]
    assert not np.isnan(np.tril(got)).any()
    # alpha = 0: A (NaN) is not read, C <- beta C on the triangle
    A[:] = np.nan
    _, C = _syrk_case("U", "T", n, k, 0.0, 2.0, seed=7)
    Ad, Cd = _dev(A), _dev(C)
    gb.ssyrk_raw("U", "N", n, k, 0.0, Ad.data_ptr(), A.shape[0], 2.0, Cd.data_ptr(), C.shape[0])
    torch.cuda.synchronize()
    got = gb.to_fortran(Cd)[:n, :n]
    iu = np.triu_indices(n)
    assert np.array_equal(got[iu], np.float32(2.0) * C[:n, :n][iu])
    # argument errors (BLAS positions)
    assert gb.ssyrk_raw("X", "N", 4, 4, 1.0, 0, 4, 0.0, 0, 4, check=False) == -1
    assert gb.ssyrk_raw("L", "N", 4, 4, 1.0, 0, 3, 0.0, 0, 4, check=False) == -7
    assert gb.ssyrk_raw("L", "T", 4, 6, 1.0, 0, 5, 0.0, 0, 4, check=False) == -7
    assert gb.ssyrk_raw("L", "N", 4, 4, 1.0, 0, 4, 0.0, 0, 3, check=False) == -10
    assert gb.ssyrk_raw("L", "N", 0, 4, 1.0, 0, 1, 0.0, 0, 1, check=False) == _lib.GB_OK


# ------------------------------------------------------------------ STRSM --

def _trsm_case(side, uplo, diag, m, n, seed, integer=False, pad=2):
    """A well-conditioned triangular A (off-diagonal entries U(-1,1)/s, |diag|
    in [1, 2]) or an integer one with a +-1 diagonal; garbage outside the
    triangle and on a unit diagonal (never read)."""
    rng = np.random.default_rng(seed)
    s = m if side == "L" else n
    lda = s + pad
    A = np.zeros((lda, s), order="F")
    if integer:
        T = rng.integers(-1, 2, (s, s)).astype(np.float64)
        np.fill_diagonal(T, rng.choice([-1.0, 1.0], s))
    else:
        T = rng.uniform(-1, 1, (s, s)) / s
        np.fill_diagonal(T, rng.uniform(1, 2, s) * rng.choice([-1, 1], s))
    i, j = np.indices((s, s))
    T[(i < j) if uplo == "L" else (i > j)] = np.nan
    if diag == "U":
        np.fill_diagonal(T, np.nan)
    A[:s, :s] = T
    A[s:, :] = wl.CANARY
    return np.asfortranarray(A, dtype=np.float32)


def _residual_check(side, uplo, trans, diag, m, n, alpha, A, B0, X, algo):
    s = m if side == "L" else n
    T = blas3.op_triangular(uplo, trans, diag, A, s)
    Xd = X.astype(np.float64)
    R = (T @ Xd if side == "L" else Xd @ T) - alpha * B0[:m, :n].astype(np.float64)
    absT = np.abs(T)
    mag = absT @ np.abs(Xd) if side == "L" else np.abs(Xd) @ absT
    depth = max(0, int(np.ceil(np.log2(max(s, 1) / 128))))
    extra = split_extra(_resolve(algo, 128) if algo == "auto" else algo, 128)
    tol = ((2 * s + 2) * U + depth * extra) * mag + 2 * U * np.abs(alpha * B0[:m, :n]) + 1e-38
    assert np.all(np.abs(R) <= tol), float(np.max(np.abs(R) / tol))


@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
@pytest.mark.parametrize("m,n", [(1, 1), (100, 70), (129, 257), (300, 130), (700, 90), (1100, 45)])
def test_strsm_residual(m, n, side, uplo, trans, diag):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    A = _trsm_case(side, uplo, diag, m, n, seed=m + 3 * n)
    rng = np.random.default_rng(m * n)
    B = wl.uniform(rng, m, n, m + 1, pad=wl.CANARY)
    Ad, Bd = _dev(A), _dev(B)
    alpha = 0.75
    gb.strsm_raw(side, uplo, trans, diag, m, n, alpha, Ad.data_ptr(), A.shape[0], Bd.data_ptr(),
                 B.shape[0], algo="auto")
    torch.cuda.synchronize()
    got = gb.to_fortran(Bd)
    assert np.all(got[m:, :] == wl.CANARY)
    _residual_check(side, uplo, trans, diag, m, n, alpha, A, B, got[:m, :n], "auto")
    X64 = blas3.strsm(side, uplo, trans, diag, m, n, alpha, A, B)
    assert np.linalg.norm(got[:m, :n] - X64) <= 1e-5 * np.linalg.norm(X64) + 1e-30


@pytest.mark.parametrize("algo", ("simt", "tf32x3", "bf16x3", "bf16x9"))
@pytest.mark.parametrize("side,uplo,trans,diag", [("L", "L", "N", "N"), ("R", "U", "T", "U")])
def test_strsm_algorithms(side, uplo, trans, diag, algo):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, n = 400, 300
    A = _trsm_case(side, uplo, diag, m, n, seed=11)
    rng = np.random.default_rng(12)
    B = wl.uniform(rng, m, n, m)
    Ad, Bd = _dev(A), _dev(B)
    gb.strsm_raw(side, uplo, trans, diag, m, n, -1.5, Ad.data_ptr(), A.shape[0], Bd.data_ptr(),
                 B.shape[0], algo=algo)
    torch.cuda.synchronize()
    _residual_check(side, uplo, trans, diag, m, n, -1.5, A, B, gb.to_fortran(Bd)[:m, :n], algo)


@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_strsm_integer_exact(side, uplo, trans, diag):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, n = 300, 200
    A = _trsm_case(side, uplo, diag, m, n, seed=13, integer=True)
    rng = np.random.default_rng(14)
    X = rng.integers(-2, 3, (m, n)).astype(np.float64)
    s = m if side == "L" else n
    T = blas3.op_triangular(uplo, trans, diag, A, s)
    Bm = T @ X if side == "L" else X @ T
    assert np.abs(Bm).max() < 2 ** 24
    B = np.asfortranarray(Bm, dtype=np.float32)
    Ad, Bd = _dev(A), _dev(B)
    gb.strsm_raw(side, uplo, trans, diag, m, n, 1.0, Ad.data_ptr(), A.shape[0], Bd.data_ptr(),
                 m, algo="auto")
    torch.cuda.synchronize()
    assert np.array_equal(gb.to_fortran(Bd)[:m, :n], X.astype(np.float32))


def test_strsm_special_cases():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, n = 150, 40
    A = np.asfortranarray(np.full((m, m), np.nan, dtype=np.float32))
    B = np.asfortranarray(np.full((m, n), np.nan, dtype=np.float32))
    Ad, Bd = _dev(A), _dev(B)
    gb.strsm_raw("L", "L", "N", "N", m, n, 0.0, Ad.data_ptr(), m, Bd.data_ptr(), m)
    torch.cuda.synchronize()
    assert np.array_equal(gb.to_fortran(Bd), np.zeros((m, n), dtype=np.float32))
    assert gb.strsm_raw("X", "L", "N", "N", 4, 4, 1.0, 0, 4, 0, 4, check=False) == -1
    assert gb.strsm_raw("L", "X", "N", "N", 4, 4, 1.0, 0, 4, 0, 4, check=False) == -2
    assert gb.strsm_raw("L", "L", "X", "N", 4, 4, 1.0, 0, 4, 0, 4, check=False) == -3
    assert gb.strsm_raw("L", "L", "N", "X", 4, 4, 1.0, 0, 4, 0, 4, check=False) == -4
    assert gb.strsm_raw("L", "L", "N", "N", 4, 4, 1.0, 0, 3, 0, 4, check=False) == -9
    assert gb.strsm_raw("R", "L", "N", "N", 4, 6, 1.0, 0, 5, 0, 4, check=False) == -9
    assert gb.strsm_raw("L", "L", "N", "N", 4, 4, 1.0, 0, 4, 0, 3, check=False) == -11


def test_strsm_workspace_rules():
    """The workspace holds the GEMM updates' area and one prepared block per
    256 rows of A's diagonal: too small or not 16-byte aligned is refused
    before any launch, and B is untouched."""
    torch = torch_gpu()
    import ctypes
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.api.default_handle()
    m, n = 300, 50
    A = _trsm_case("L", "L", "N", m, n, seed=21)
    B = wl.uniform(np.random.default_rng(22), m, n, m)
    Ad, Bd = _dev(A), _dev(B)
    need = ctypes.c_size_t(0)
    assert h.lib.gb_strsm_workspace_size(_lib.ALGOS["simt"], b"L", b"L", b"N", b"N", m, n,
                                         ctypes.byref(need)) == _lib.GB_OK
    assert need.value >= 2 * 140288                     # two diagonal blocks, even for SIMT
    ws = torch.empty(need.value + 16, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for ptr, size in ((0, 0), (ws.data_ptr(), need.value - 1), (ws.data_ptr() + 4, need.value)):
        rc = h.lib.gb_strsm(h.h, _lib.ALGOS["simt"], b"L", b"L", b"N", b"N", m, n, 1.0,
                            Ad.data_ptr(), A.shape[0], Bd.data_ptr(), m, ptr, size, s)
        assert rc == _lib.GB_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert np.array_equal(gb.to_fortran(Bd), B)
    rc = h.lib.gb_strsm(h.h, _lib.ALGOS["simt"], b"L", b"L", b"N", b"N", m, n, 1.0,
                        Ad.data_ptr(), A.shape[0], Bd.data_ptr(), m, ws.data_ptr() + 16,
                        need.value, s)
    assert rc == _lib.GB_OK
    torch.cuda.synchronize()
    _residual_check("L", "L", "N", "N", m, n, 1.0, A, B, gb.to_fortran(Bd)[:m, :n], "simt")
