"""CPU oracle for two more Level-3 BLAS operations on the SGEMM core, in double
precision: SSYRK (symmetric rank-k update) and STRSM (triangular solve with
many right-hand sides).

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`).

The paper builds its SGEMM behind the Level-3 BLAS interface (Sec. 1), whose
other routines (and LAPACK above them) are written on top of GEMM. The
definitions, for column-major float32 inputs and BLAS argument conventions:

  ssyrk   C <- alpha op(A) op(A)^T + beta C on the `uplo` triangle of the
          n x n matrix C only (op(A) = A, n x k, for 'N'; A^T, A k x n, for
          'T'); the other triangle is not referenced. As for SGEMM, C is not
          read when beta = 0 and A is not read when alpha = 0 or k = 0.
          Written out with the SGEMM oracle (B = A), keeping the triangle.
  strsm   X with op(A) X = alpha B (side 'L', A m x m) or X op(A) = alpha B
          (side 'R', A n x n), A triangular ('U' or 'L'), unit diagonal
          assumed (not read) for diag 'U'; X overwrites B. B is first scaled
          by alpha, then solved by plain substitution in FP64 (one row of X at
          a time for side 'L', one column for side 'R', in dependency order).
          alpha = 0 gives X = 0 without reading A or B.
"""
from __future__ import annotations

import numpy as np

from . import sgemm as _sgemm


def _tri_mask(n, uplo):
    i, j = np.indices((n, n))
    return (i >= j) if uplo in "Ll" else (i <= j)


def ssyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc):
    """Return (C64, D) over the full n x n shape; entries outside the `uplo`
    triangle are NaN (they are not part of the result). A and C are Fortran
    float32 arrays with leading dimensions lda and ldc."""
    tb = "T" if trans in "Nn" else "N"
    C64, D = _sgemm(trans.upper(), tb, n, n, k, alpha, A, lda, A, lda, beta, C, ldc)
    mask = _tri_mask(n, uplo)
    C64 = np.where(mask, C64, np.nan)
    D = np.where(mask, D, np.nan)
    return C64, D


def op_triangular(uplo, trans, diag, A, s):
    """op(A) of the s x s triangular matrix stored in A (float64), with the
    unreferenced triangle zeroed and a unit diagonal for diag 'U'."""
    T = np.array(A[:s, :s], dtype=np.float64)
    T = np.where(_tri_mask(s, uplo), T, 0.0)
    if diag in "Uu":
        np.fill_diagonal(T, 1.0)
    return T.T.copy() if trans in "TtCc" else T


def strsm(side, uplo, trans, diag, m, n, alpha, A, B):
    """X (m x n, float64) solving op(A) X = alpha B or X op(A) = alpha B by
    substitution. A and B are float32 arrays (A s x s with s = m or n)."""
    if m == 0 or n == 0:
        return np.zeros((m, n))
    if alpha == 0.0:
        return np.zeros((m, n))
    left = side in "Ll"
    s = m if left else n
    T = op_triangular(uplo, trans, diag, A, s)
    R = float(alpha) * np.array(B[:m, :n], dtype=np.float64)
    # op(A) is lower triangular iff A is lower and not transposed, or upper
    # and transposed
    lower = (uplo in "Ll") != (trans in "TtCc")
    X = np.zeros((m, n))
    if left:
        # row i of X: (R_i - T[i, done] X[done]) / T[i, i]
        order = range(m) if lower else range(m - 1, -1, -1)
        for i in order:
            done = slice(0, i) if lower else slice(i + 1, m)
            X[i] = (R[i] - T[i, done] @ X[done]) / T[i, i]
    else:
        # column j of X: (R[:, j] - X[:, done] T[done, j]) / T[j, j]
        upper = not lower
        order = range(n) if upper else range(n - 1, -1, -1)
        for j in order:
            done = slice(0, j) if upper else slice(j + 1, n)
            X[:, j] = (R[:, j] - X[:, done] @ T[done, j]) / T[j, j]
    return X
