"""Pins that tie the CPU oracle to the definition of SGEMM, not to itself.

The paper defines the operation only as the Level-3 BLAS SGEMM with a 2MNK
dense product (Sec. 1) and prints no numeric example, so the oracle is pinned
by exact rational brute force, closed forms (identity, permutation, rank-1,
hand-worked examples in tests/golden/), BLAS special cases (alpha = 0,
beta = 0, K = 0), transpose equivalence, exact integer arithmetic and an
independent library product. Each pin is a function of an `sgemm` callable
so that `test_pins_catch_planted_mistakes` can run the same pins against
deliberately broken copies of the oracle (built on the CPU) and show that
every planted mistake fails at least one of them.
"""
import json
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


def _fortran(mat_rows, ld=None):
    a = np.array(mat_rows, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return wl.embed(a.astype(np.float32), ld or max(a.shape[0], 1), np.nan)


def _nan(rows, cols):
    return np.full((rows, cols), np.nan, dtype=np.float32, order="F")


def _op(trans, X, rows, cols):
    """op(X) as a dense float64 (rows x cols) matrix, written out elementwise."""
    out = np.zeros((rows, cols))
    for i in range(rows):
        for j in range(cols):
            out[i, j] = X[i, j] if trans == "N" else X[j, i]
    return out


# ---------------------------------------------------------------- pins -----

def pin_golden(sgemm):
    """Hand-worked closed-form examples (tests/golden/hand_examples.json)."""
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        A = _fortran(c["A"], ld=len(c["A"]) + 2)
        B = _fortran(c["B"], ld=len(c["B"]) + 1)
        Cv = [[float(x) for x in row] for row in c["C"]]
        C = _fortran(Cv, ld=c["m"] + 3)
        C64, D = sgemm(c["ta"], c["tb"], c["m"], c["n"], c["k"], c["alpha"], A, A.shape[0],
                       B, B.shape[0], c["beta"], C, C.shape[0])
        if not (np.array_equal(C64, np.array(c["expected"], dtype=np.float64))
                and np.array_equal(D, np.array(c["expected_D"], dtype=np.float64))):
            return False
    return True


def pin_fraction_bruteforce(sgemm, seed=11):
    """Exact rational arithmetic on tiny non-square shapes, all transposes,
    padded leading dimensions and random alpha/beta."""
    rng = np.random.default_rng(seed)
    for ta, tb in TRANS:
        for (m, n, k) in [(1, 1, 1), (2, 3, 4), (5, 2, 3), (4, 6, 5), (3, 5, 6), (6, 4, 2)]:
            p = wl.make_problem(ta, tb, m, n, k, rng.uniform(-2, 2), rng.uniform(-2, 2),
                                rng=rng, ld_pad=int(rng.integers(0, 3)))
            C64, D = sgemm(ta, tb, m, n, k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc)
            ar, ac = wl.stored_shape(ta, m, k)
            br, bc = wl.stored_shape(tb, k, n)
            Ax, Bx = p.A[:ar, :ac], p.B[:br, :bc]
            for i in range(m):
                for j in range(n):
                    s = Fraction(0)
                    sa = Fraction(0)
                    for q in range(k):
                        a = Fraction(float(Ax[i, q] if ta == "N" else Ax[q, i]))
                        b = Fraction(float(Bx[q, j] if tb == "N" else Bx[j, q]))
                        s += a * b
                        sa += abs(a) * abs(b)
                    cij = Fraction(float(p.C[i, j]))
                    exact = Fraction(p.alpha) * s + Fraction(p.beta) * cij
                    dex = abs(Fraction(p.alpha)) * sa + abs(Fraction(p.beta)) * abs(cij)
                    tol = (k + 3) * 2.0 ** -53 * float(dex)
                    if abs(C64[i, j] - float(exact)) > tol or abs(D[i, j] - float(dex)) > tol:
                        return False
    return True


def pin_identity_permutation(sgemm, seed=12):
    """A = I gives C = alpha*op(B) + beta*C exactly (alpha=1, beta=0 and
    alpha=2, beta=0.5 both exact for these values); a permutation matrix
    permutes rows of op(B) exactly; B = I gives op(A)."""
    rng = np.random.default_rng(seed)
    m, n = 7, 5
    for ta, tb in TRANS:
        I = _fortran(np.eye(m))
        Bp = wl.make_problem("N", tb, m, n, m, 1.0, 0.0, rng=rng)
        opB = _op(tb, Bp.B, m, n)
        C = wl.uniform(rng, m, n)
        C64, _ = sgemm(ta, tb, m, n, m, 2.0, I, m, Bp.B, Bp.ldb, 0.5, C, m)
        if not np.array_equal(C64, 2.0 * opB + 0.5 * C.astype(np.float64)):
            return False
        perm = rng.permutation(m)
        P = np.zeros((m, m))
        P[np.arange(m), perm] = 1.0          # (P X)[i] = X[perm[i]]
        Pst = P if ta == "N" else P.T
        C64, _ = sgemm(ta, tb, m, n, m, 1.0, _fortran(Pst), m, Bp.B, Bp.ldb, 0.0, _nan(m, n), m)
        if not np.array_equal(C64, opB[perm, :]):
            return False
        # B = I: C = op(A)
        Ap = wl.make_problem(ta, "N", m, n, n, 1.0, 0.0, rng=rng)
        opA = _op(ta, Ap.A, m, n)
        C64, _ = sgemm(ta, tb, m, n, n, 1.0, Ap.A, Ap.lda, _fortran(np.eye(n)), n, 0.0, _nan(m, n), m)
        if not np.array_equal(C64, opA):
            return False
    return True


def pin_rank1(sgemm, seed=13):
    """K = 1: C_ij = alpha*a_i*b_j + beta*c_ij. A = x 1^T, B = 1 y^T with
    small integers: (AB)_ij = K x_i y_j exactly."""
    rng = np.random.default_rng(seed)
    m, n = 6, 9
    for ta, tb in TRANS:
        p = wl.make_problem(ta, tb, m, n, 1, -1.25, 0.75, rng=rng)
        x = p.A[:m, 0] if ta == "N" else p.A[0, :m]
        y = p.B[0, :n] if tb == "N" else p.B[:n, 0]
        want = (-1.25 * np.outer(x.astype(np.float64), y.astype(np.float64))
                + 0.75 * p.C[:m, :n].astype(np.float64))
        C64, _ = sgemm(ta, tb, m, n, 1, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc)
        if np.max(np.abs(C64 - want)) > 4 * 2.0 ** -53 * np.max(np.abs(want)):
            return False
        k = 37
        xi = rng.integers(-9, 10, size=m).astype(np.float64)
        yi = rng.integers(-9, 10, size=n).astype(np.float64)
        Aop, Bop = np.outer(xi, np.ones(k)), np.outer(np.ones(k), yi)
        A = _fortran(Aop if ta == "N" else Aop.T)
        B = _fortran(Bop if tb == "N" else Bop.T)
        C64, _ = sgemm(ta, tb, m, n, k, 1.0, A, A.shape[0], B, B.shape[0], 0.0, _nan(m, n), m)
        if not np.array_equal(C64, k * np.outer(xi, yi)):
            return False
    return True


def pin_blas_special_cases(sgemm, seed=14):
    """alpha = 0 reads neither A nor B (NaN-filled); beta = 0 never reads C
    (NaN-filled); K = 0 gives beta*C."""
    rng = np.random.default_rng(seed)
    m, n, k = 5, 4, 3
    for ta, tb in TRANS:
        ar, ac = wl.stored_shape(ta, m, k)
        br, bc = wl.stored_shape(tb, k, n)
        nanA = np.full((ar, ac), np.nan, dtype=np.float32, order="F")
        nanB = np.full((br, bc), np.nan, dtype=np.float32, order="F")
        C = wl.uniform(rng, m, n)
        C64, D = sgemm(ta, tb, m, n, k, 0.0, nanA, ar, nanB, br, -0.5, C, m)
        if not np.array_equal(C64, -0.5 * C.astype(np.float64)):
            return False
        if not np.array_equal(D, 0.5 * np.abs(C.astype(np.float64))):
            return False
        p = wl.make_problem(ta, tb, m, n, k, 1.0, 0.0, rng=rng)
        nanC = np.full((m, n), np.nan, dtype=np.float32, order="F")
        C64, _ = sgemm(ta, tb, m, n, k, 1.0, p.A, p.lda, p.B, p.ldb, 0.0, nanC, m)
        if not np.all(np.isfinite(C64)):
            return False
        C64, _ = sgemm(ta, tb, m, n, 0, 1.0, nanA, max(ar, 1), nanB, max(br, 1), 3.0, C, m)
        if not np.array_equal(C64, 3.0 * C.astype(np.float64)):
            return False
    return True


def pin_transpose_equivalence(sgemm, seed=15):
    """oracle('T', A) equals oracle('N', explicit A^T copy) bit for bit (same
    per-element summation order), and likewise for B."""
    rng = np.random.default_rng(seed)
    m, n, k = 9, 7, 11
    p = wl.make_problem("N", "N", m, n, k, 1.5, -0.5, rng=rng, ld_pad=3)
    ref, refD = sgemm("N", "N", m, n, k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc)
    At = wl.embed(np.ascontiguousarray(p.A[:m, :k].T), k + 2, np.nan)
    Bt = wl.embed(np.ascontiguousarray(p.B[:k, :n].T), n + 1, np.nan)
    for ta, tb, A, lda, B, ldb in [("T", "N", At, k + 2, p.B, p.ldb),
                                   ("N", "T", p.A, p.lda, Bt, n + 1),
                                   ("T", "T", At, k + 2, Bt, n + 1)]:
        got, gotD = sgemm(ta, tb, m, n, k, p.alpha, A, lda, B, ldb, p.beta, p.C, p.ldc)
        if not (np.array_equal(got, ref) and np.array_equal(gotD, refD)):
            return False
    return True


def pin_integer_exact(sgemm, seed=16):
    """Integer inputs in {-8..8}: every partial sum is an integer far below
    2^53, so the result equals exact integer arithmetic."""
    rng = np.random.default_rng(seed)
    for ta, tb in TRANS:
        m, n, k = 13, 10, 97
        p = wl.make_problem(ta, tb, m, n, k, 1.0, 0.5, rng=rng, dist="int", ld_pad=2)
        ar, ac = wl.stored_shape(ta, m, k)
        br, bc = wl.stored_shape(tb, k, n)
        Ai = p.A[:ar, :ac].astype(np.int64)
        Bi = p.B[:br, :bc].astype(np.int64)
        Ai = Ai if ta == "N" else Ai.T
        Bi = Bi if tb == "N" else Bi.T
        exact = (Ai @ Bi).astype(np.float64) + 0.5 * p.C[:m, :n].astype(np.float64)
        C64, D = sgemm(ta, tb, m, n, k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc)
        if not np.array_equal(C64, exact):
            return False
        dex = (np.abs(Ai) @ np.abs(Bi)).astype(np.float64) + 0.5 * np.abs(p.C[:m, :n].astype(np.float64))
        if not np.array_equal(D, dex):
            return False
    return True


def pin_library_product(sgemm, seed=17):
    """numpy's float64 matmul (different summation order) agrees within
    K * 2^-53 * D on larger non-square shapes."""
    rng = np.random.default_rng(seed)
    for ta, tb in TRANS:
        m, n, k = 67, 45, 130
        p = wl.make_problem(ta, tb, m, n, k, 0.75, -1.5, rng=rng, ld_pad=5)
        ar, ac = wl.stored_shape(ta, m, k)
        br, bc = wl.stored_shape(tb, k, n)
        Ax = p.A[:ar, :ac].astype(np.float64)
        Bx = p.B[:br, :bc].astype(np.float64)
        Ax = Ax if ta == "N" else Ax.T
        Bx = Bx if tb == "N" else Bx.T
        want = 0.75 * (Ax @ Bx) - 1.5 * p.C[:m, :n].astype(np.float64)
        dwant = 0.75 * (np.abs(Ax) @ np.abs(Bx)) + 1.5 * np.abs(p.C[:m, :n].astype(np.float64))
        C64, D = sgemm(ta, tb, m, n, k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc)
        tol = (k + 4) * 2.0 ** -53 * dwant
        if not (np.all(np.abs(C64 - want) <= tol) and np.all(np.abs(D - dwant) <= tol)):
            return False
    return True


def pin_column_subset(sgemm, seed=18):
    """Selecting output columns returns exactly those columns of the full result."""
    rng = np.random.default_rng(seed)
    m, n, k = 20, 33, 17
    for ta, tb in TRANS:
        p = wl.make_problem(ta, tb, m, n, k, 1.0, 1.0, rng=rng, ld_pad=1)
        full, fullD = sgemm(ta, tb, m, n, k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc)
        cols = np.array([32, 0, 5, 5, 17])
        sub, subD = sgemm(ta, tb, m, n, k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc,
                          cols=cols)
        if not (np.array_equal(sub, full[:, cols]) and np.array_equal(subD, fullD[:, cols])):
            return False
    return True


PINS = [pin_golden, pin_fraction_bruteforce, pin_identity_permutation, pin_rank1,
        pin_blas_special_cases, pin_transpose_equivalence, pin_integer_exact,
        pin_library_product, pin_column_subset]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    assert pin(oracle.sgemm)


def test_oracle_threads_do_not_change_results():
    p = wl.make_problem("T", "N", 70, 40, 300, 1.5, -0.5, seed=5, ld_pad=7)
    a = oracle.sgemm("T", "N", 70, 40, 300, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc,
                     nthreads=1)
    b = oracle.sgemm("T", "N", 70, 40, 300, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C, p.ldc,
                     nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_oracle_rejects_bad_arguments():
    A = np.zeros((1, 1), dtype=np.float32, order="F")
    with pytest.raises(ValueError):
        oracle.sgemm("X", "N", 1, 1, 1, 1.0, A, 1, A, 1, 0.0, None, 1)
    with pytest.raises(ValueError):
        oracle.sgemm("N", "N", -1, 1, 1, 1.0, A, 1, A, 1, 0.0, None, 1)


# ------------------------------------------------- dgemm and the report ----

def test_dgemm_matches_exact_rationals():
    rng = np.random.default_rng(19)
    for ta, tb in TRANS:
        m, n, k = 3, 4, 5
        A = np.asfortranarray(rng.normal(size=wl.stored_shape(ta, m, k)))
        B = np.asfortranarray(rng.normal(size=wl.stored_shape(tb, k, n)))
        C = np.asfortranarray(rng.normal(size=(m, n)))
        got = oracle.dgemm(ta, tb, m, n, k, 0.5, A, A.shape[0], B, B.shape[0], 2.0, C, m)
        opA = _op(ta, A, m, k)
        opB = _op(tb, B, k, n)
        for i in range(m):
            for j in range(n):
                s = sum(Fraction(opA[i, q]) * Fraction(opB[q, j]) for q in range(k))
                ex = Fraction(0.5) * s + Fraction(2.0) * Fraction(C[i, j])
                assert abs(got[i, j] - float(ex)) <= 1e-14 * (1 + abs(float(ex)))


def test_err_report_definition():
    C64 = np.array([[1.0, 2.0], [3.0, 0.0]], order="F")
    D = np.array([[1.0, 2.0], [4.0, 0.0]], order="F")
    k = 4
    b = 2 * k * 2.0 ** -24
    C = np.array([[1.0 + b / 2, 2.0], [3.0 - 8 * b, 0.0]], dtype=np.float64, order="F")
    r = oracle.err_report(C, C64, D, k)
    # ratios: 0.5, 0, 2, 0 (the bound-zero element matches exactly)
    assert r["max_ratio"] == pytest.approx(2.0)
    assert r["median_ratio"] == 0.0            # sorted (0, 0, 0.5, 2): rank 1
    assert r["n_fail"] == 1 and r["count"] == 4
    want = np.sqrt((b / 2) ** 2 + (8 * b) ** 2) / np.sqrt(1 + 4 + 9)
    assert r["normwise"] == pytest.approx(want, rel=1e-12)
    C[1, 1] = 1e-30                            # nonzero error on a zero bound
    assert oracle.err_report(C, C64, D, k)["max_ratio"] == np.inf
    assert oracle.bound(np.array([1.0]), 0)[0] == 2.0 * 2.0 ** -24


# ---------------------------------------------------- mutation check -------

MUTANTS = {
    "dropped_beta_term": ("        v += beta * c;\n", "\n"),
    "wrong_sign": ("s[i] += a * b;", "s[i] -= a * b;"),
    "transposed_A_index": ("return is_n(ta) ? A[i + p * lda] : A[p + i * lda];",
                           "return is_n(ta) ? A[p + i * lda] : A[i + p * lda];"),
    "wrong_B_index": ("return is_n(tb) ? B[p + j * ldb] : B[j + p * ldb];",
                      "return is_n(tb) ? B[p + j * ldb] : B[p + j * ldb];"),
    "alpha_dropped": ("    double v = alpha * s;\n", "    double v = s;\n"),
    "cols_ignored": ("int64_t j = cols ? cols[q] : q;", "int64_t j = q;"),
    "off_by_one_k": ("for (int64_t p = 0; p < k; ++p) {\n                        double b",
                     "for (int64_t p = 1; p < k; ++p) {\n                        double b"),
    "reads_C_when_beta0": ("    if (beta != 0.0) {\n        double c", "    if (1) {\n        double c"),
    "abs_dropped_in_D": ("sai += fabs(a) * fabs(b);", "sai += a * b;"),
    "float_accumulation": ("double si = 0.0, sai = 0.0;", "float si = 0.0f; double sai = 0.0;"),
}


def _build_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src, f"mutation anchor for {name} not found"
    src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", str(c),
                    "-o", str(so), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(name, tmp_path, monkeypatch):
    """Each planted mistake in a copy of the oracle fails at least one pin."""
    import ctypes
    so = _build_mutant(name, tmp_path)
    lib = ctypes.CDLL(so)
    real = oracle._load()
    lib.oracle_sgemm.argtypes = real.oracle_sgemm.argtypes
    lib.oracle_sgemm.restype = ctypes.c_int
    monkeypatch.setattr(oracle, "_lib", lib)
    failed = []
    for pin in PINS:
        try:
            ok = pin(oracle.sgemm)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
