"""Pins for the SSYRK and STRSM oracles (oracle/blas3.py), fixed by exact
arithmetic and closed forms:

  * exact rational brute force (fractions) on tiny shapes, every flag set;
  * SSYRK: a rank-1 update has the closed form alpha a a^T + beta C, the full
    product A A^T is exactly symmetric, the other triangle is not produced;
  * STRSM: op(A) = I gives alpha B; a diagonal op(A) gives alpha B / d; an
    integer unit-triangular op(A) times an integer X recovers X exactly, for
    all 16 combinations of side, uplo, trans and diag;
  * alpha = 0 gives X = 0 without reading NaN-filled A and B.

Planted mistakes (uplo swapped for side 'L', the diagonal read for diag 'U',
alpha dropped, the wrong triangle kept by SSYRK) each fail a pin.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import blas3

COMBOS = list(itertools.product("LR", "LU", "NT", "NU"))


def _f32(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float32))


def _tri_exact(uplo, trans, diag, A, s):
    T = [[Fraction(0)] * s for _ in range(s)]
    for i in range(s):
        for j in range(s):
            inside = i >= j if uplo == "L" else i <= j
            if inside:
                T[i][j] = Fraction(float(A[i, j]))
        if diag == "U":
            T[i][i] = Fraction(1)
    if trans == "T":
        T = [[T[j][i] for j in range(s)] for i in range(s)]
    return T


def _solve_exact(side, uplo, trans, diag, m, n, alpha, A, B):
    """X by Gaussian elimination in exact rationals (no ordering assumption)."""
    s = m if side == "L" else n
    T = _tri_exact(uplo, trans, diag, A, s)
    R = [[Fraction(float(alpha)) * Fraction(float(B[i, j])) for j in range(n)] for i in range(m)]
    if side == "R":          # X T = R  <=>  T^T X^T = R^T
        T = [[T[j][i] for j in range(s)] for i in range(s)]
        R = [[R[i][j] for i in range(m)] for j in range(n)]
    cols = len(R[0])
    M = [T[i][:] + R[i][:] for i in range(s)]
    for c in range(s):                       # Gauss-Jordan on a nonsingular T
        p = next(r for r in range(c, s) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(s):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    X = [[M[i][s + j] for j in range(cols)] for i in range(s)]
    if side == "R":
        X = [[X[j][i] for j in range(n)] for i in range(m)]
    return np.array([[float(v) for v in row] for row in X])


def _tri_problem(rng, side, uplo, diag, m, n, integer=False):
    s = m if side == "L" else n
    if integer:
        A = rng.integers(-2, 3, (s, s)).astype(np.float64)
        np.fill_diagonal(A, rng.choice([-1.0, 1.0], s))
    else:
        A = rng.uniform(-1, 1, (s, s))
        np.fill_diagonal(A, rng.uniform(1.5, 3.0, s) * rng.choice([-1, 1], s))
    # the unreferenced triangle holds garbage that must not be read
    i, j = np.indices((s, s))
    outside = (i < j) if uplo == "L" else (i > j)
    A[outside] = 1e30
    if diag == "U":
        np.fill_diagonal(A, 7e29)
    B = rng.integers(-3, 4, (m, n)).astype(np.float64) if integer else rng.uniform(-1, 1, (m, n))
    return _f32(A), _f32(B)


@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_strsm_brute_force_tiny(side, uplo, trans, diag):
    rng = np.random.default_rng(COMBOS.index((side, uplo, trans, diag)))
    for (m, n) in ((1, 1), (3, 2), (2, 4), (4, 3)):
        A, B = _tri_problem(rng, side, uplo, diag, m, n)
        X = blas3.strsm(side, uplo, trans, diag, m, n, 0.75, A, B)
        want = _solve_exact(side, uplo, trans, diag, m, n, np.float32(0.75), A, B)
        assert np.allclose(X, want, rtol=1e-13, atol=1e-13), (m, n)


@pytest.mark.parametrize("side,uplo,trans,diag", COMBOS)
def test_strsm_integer_recovery(side, uplo, trans, diag):
    rng = np.random.default_rng(7)
    m, n = 9, 7
    A, _ = _tri_problem(rng, side, uplo, diag, m, n, integer=True)
    X = rng.integers(-3, 4, (m, n)).astype(np.float64)
    s = m if side == "L" else n
    T = blas3.op_triangular(uplo, trans, diag, A, s)
    B = _f32(T @ X if side == "L" else X @ T)
    got = blas3.strsm(side, uplo, trans, diag, m, n, 1.0, A, B)
    assert np.array_equal(got, X)


def test_strsm_identity_and_diagonal():
    rng = np.random.default_rng(8)
    B = _f32(rng.uniform(-1, 1, (5, 6)))
    eye = _f32(np.eye(5))
    for uplo, trans in itertools.product("LU", "NT"):
        assert np.array_equal(blas3.strsm("L", uplo, trans, "N", 5, 6, 1.5, eye, B),
                              1.5 * B.astype(np.float64))
    d = np.array([2.0, -4.0, 0.5, 8.0, -1.0, 0.25])
    Dg = _f32(np.diag(d))
    X = blas3.strsm("R", "U", "N", "N", 5, 6, 1.0, Dg, B)
    assert np.array_equal(X, B.astype(np.float64) / d[None, :])


def test_strsm_alpha_zero_reads_nothing():
    A = _f32(np.full((4, 4), np.nan))
    B = _f32(np.full((4, 3), np.nan))
    assert np.array_equal(blas3.strsm("L", "L", "N", "N", 4, 3, 0.0, A, B), np.zeros((4, 3)))


@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_ssyrk_brute_force_and_symmetry(uplo, trans):
    rng = np.random.default_rng(9)
    n, k = 4, 3
    A = _f32(rng.uniform(-1, 1, (n, k) if trans == "N" else (k, n)))
    C = _f32(rng.uniform(-1, 1, (n, n)))
    C64, D = blas3.ssyrk(uplo, trans, n, k, 1.25, A, A.shape[0], -0.5, C, n)
    opA = [[Fraction(float(A[i, p] if trans == "N" else A[p, i])) for p in range(k)]
           for i in range(n)]
    for i in range(n):
        for j in range(n):
            inside = i >= j if uplo == "L" else i <= j
            if not inside:
                assert np.isnan(C64[i, j])
                continue
            want = Fraction(1.25) * sum(opA[i][p] * opA[j][p] for p in range(k)) + \
                Fraction(-0.5) * Fraction(float(C[i, j]))
            # FP64 accumulation of k products and the beta term: (k + 2) 2^-53 D
            assert abs(C64[i, j] - float(want)) <= (k + 2) * 2.0 ** -53 * D[i, j]
    full, _ = oracle.sgemm(trans, "T" if trans == "N" else "N", n, n, k, 1.0, A, A.shape[0],
                           A, A.shape[0], 0.0, None, n)
    assert np.array_equal(full, full.T)


def test_ssyrk_rank_one_closed_form():
    a = _f32([[1.0], [-2.0], [3.0]])
    C = _f32(np.arange(9, dtype=np.float64).reshape(3, 3))
    C64, _ = blas3.ssyrk("U", "N", 3, 1, 2.0, a, 3, 0.5, C, 3)
    want = 2.0 * (a @ a.T).astype(np.float64) + 0.5 * C
    iu = np.triu_indices(3)
    assert np.array_equal(C64[iu], want[iu])


# ------------------------------------------------------ planted mistakes --

def _pins_pass():
    try:
        for c in COMBOS:
            test_strsm_brute_force_tiny(*c)
            test_strsm_integer_recovery(*c)
        test_strsm_identity_and_diagonal()
        test_strsm_alpha_zero_reads_nothing()
        for c in itertools.product("LU", "NT"):
            test_ssyrk_brute_force_and_symmetry(*c)
        test_ssyrk_rank_one_closed_form()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mistake", ["swapped_uplo_left", "unit_diag_read", "no_alpha",
                                     "wrong_triangle"])
def test_planted_mistakes_fail_a_pin(monkeypatch, mistake):
    assert _pins_pass()
    orig_op, orig_mask, orig_strsm = blas3.op_triangular, blas3._tri_mask, blas3.strsm
    if mistake == "swapped_uplo_left":
        monkeypatch.setattr(blas3, "strsm", lambda side, uplo, *a: orig_strsm(
            side, "U" if uplo == "L" else "L", *a) if side == "L" else orig_strsm(side, uplo, *a))
    elif mistake == "unit_diag_read":
        monkeypatch.setattr(blas3, "op_triangular",
                            lambda uplo, trans, diag, A, s: orig_op(uplo, trans, "N", A, s))
    elif mistake == "no_alpha":
        monkeypatch.setattr(blas3, "strsm", lambda side, uplo, trans, diag, m, n, alpha, A, B:
                            orig_strsm(side, uplo, trans, diag, m, n, 1.0 if alpha else 0.0, A, B))
    elif mistake == "wrong_triangle":
        monkeypatch.setattr(blas3, "_tri_mask", lambda n, uplo: orig_mask(
            n, "U" if uplo in "Ll" else "L"))
    assert not _pins_pass()
