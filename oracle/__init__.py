"""CPU oracle for C <- alpha*op(A)*op(B) + beta*C, in double precision.

TEST INFRASTRUCTURE ONLY. The oracle is the plain definition of the SGEMM
computation (paper Sec. 1: dense multiplication with A: M x K and B: K x N,
2MNK flops, behind the Level-3 BLAS SGEMM interface), written as a triple
loop in C (`oracle.c`) with double accumulation. Only the tests, the smoke
check and the benchmark's CPU-baseline leg use it; the CUDA library neither
imports nor links it, and it shares no code with the library.

Every function here cites what it follows:
  * `sgemm` - the definition above plus the bound denominator
    D = |alpha|*|op(A)||op(B)| + |beta|*|C| (per element);
  * `dgemm` - the same on double inputs (finite-difference checks);
  * `bound` - the per-element acceptance bound 2*max(K,1)*2^-24*D;
  * `err_report` - max and lower-median of |C - C64| / bound and the
    normwise relative error ||C - C64||_F / ||C64||_F.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

U32 = 2.0 ** -24  # FP32 unit roundoff


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                    "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, f64 = ctypes.c_int64, ctypes.c_double
            vp = ctypes.c_void_p
            lib.oracle_sgemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64,
                                         f64, vp, i64, vp, i64, f64, vp, i64,
                                         vp, i64, vp, i64, vp, i64, ctypes.c_int]
            lib.oracle_sgemm.restype = ctypes.c_int
            lib.oracle_dgemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64,
                                         f64, vp, i64, vp, i64, f64, vp, i64,
                                         vp, i64, ctypes.c_int]
            lib.oracle_dgemm.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check_f(a, dtype, name):
    if a is None:
        return
    if a.dtype != dtype or not a.flags.f_contiguous:
        raise TypeError(f"{name} must be a Fortran-ordered {dtype} array")


def sgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
          cols=None, nthreads=0):
    """Return (C64, D), each a Fortran (m, ncols) float64 array.

    A, B, C are Fortran-ordered float32 arrays holding column-major matrices
    with leading dimensions lda, ldb, ldc (C may be None when beta == 0; A and
    B may be None when alpha == 0). `cols` selects output columns (all if
    None); column q of the result is column cols[q] of the product.
    """
    lib = _load()
    for x, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_f(x, np.float32, nm)
    if cols is None:
        colsv, ncols = None, n
    else:
        colsv = np.ascontiguousarray(cols, dtype=np.int64)
        ncols = colsv.size
    C64 = np.zeros((m, ncols), dtype=np.float64, order="F")
    D = np.zeros((m, ncols), dtype=np.float64, order="F")
    rc = lib.oracle_sgemm(ta.encode(), tb.encode(), m, n, k, float(alpha),
                          _ptr(A), lda, _ptr(B), ldb, float(beta), _ptr(C), ldc,
                          _ptr(colsv), ncols, _ptr(C64), max(m, 1), _ptr(D), max(m, 1),
                          int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_sgemm failed with {rc}")
    return C64, D


def dgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=0):
    """The same definition on float64 inputs; returns a Fortran (m, n) array."""
    lib = _load()
    for x, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_f(x, np.float64, nm)
    out = np.zeros((m, n), dtype=np.float64, order="F")
    rc = lib.oracle_dgemm(ta.encode(), tb.encode(), m, n, k, float(alpha),
                          _ptr(A), lda, _ptr(B), ldb, float(beta), _ptr(C), ldc,
                          _ptr(out), max(m, 1), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_dgemm failed with {rc}")
    return out


def op(trans, X):
    """op(X) as a new array: X for 'N', X^T for 'T'/'C'."""
    return np.array(X if trans in "Nn" else X.T, order="F")


def sgemm_backward(ta, tb, alpha, A, B, beta, G):
    """Reference gradients of L = sum(G * (alpha*op(A)*op(B) + beta*C)).

    A, B, G are dense float64 arrays (A and B in their stored shapes, G is
    M x N). Differentiating the bilinear map: dL/dop(A) = alpha*G*op(B)^T,
    dL/dop(B) = alpha*op(A)^T*G, dL/dC = beta*G; the gradient of a stored
    operand is that of op(X), transposed back when X was transposed. Each
    product is one call of the double-precision triple loop.
    Returns (dA, dB, dC) as Fortran float64 arrays.
    """
    A = np.asfortranarray(A, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    G = np.asfortranarray(G, dtype=np.float64)
    opA, opB = op(ta, A), op(tb, B)
    m, k = opA.shape
    n = opB.shape[1]
    opBt = np.asfortranarray(opB.T)
    opAt = np.asfortranarray(opA.T)
    d_opA = dgemm("N", "N", m, k, n, alpha, G, max(m, 1), opBt, max(n, 1), 0.0, None, 1)
    d_opB = dgemm("N", "N", k, n, m, alpha, opAt, max(k, 1), G, max(m, 1), 0.0, None, 1)
    dA = d_opA if ta in "Nn" else np.asfortranarray(d_opA.T)
    dB = d_opB if tb in "Nn" else np.asfortranarray(d_opB.T)
    return dA, dB, np.asfortranarray(beta * G)


def bound(D, k, extra=0.0):
    """Per-element acceptance bound (2*max(K,1)*u + extra)*D, u = 2^-24.

    The stated bound is 2*K*u*D; at K = 0 the result is beta*C rounded once
    to FP32, so max(K, 1) keeps the bound defined there. `extra` adds a
    fixed relative term (the truncation of a split-precision product).
    """
    return (2.0 * max(int(k), 1) * U32 + extra) * np.asarray(D, dtype=np.float64)


def err_report(C, C64, D, k, extra=0.0):
    """Error of an FP32 result C against the double oracle (C64, D).

    ratio_ij = |C_ij - C64_ij| / bound_ij, with ratio 0 where both are 0 and
    +inf where only the bound is 0. Two NaNs, or two infinities of the same
    sign, count as agreeing (ratio 0); one non-finite side alone is +inf.
    Returns max ratio, lower median (the element of rank floor((n-1)/2) in
    ascending order), normwise ||C - C64||_F / ||C64||_F, the number of
    elements over the bound, and the element count.
    """
    c = np.asarray(C, dtype=np.float64).ravel(order="F")
    r = np.asarray(C64, dtype=np.float64).ravel(order="F")
    b = bound(np.asarray(D).ravel(order="F"), k, extra)
    fin = np.isfinite(c) & np.isfinite(r)
    same_nf = (~fin) & ((np.isnan(c) & np.isnan(r)) | (c == r))
    with np.errstate(invalid="ignore"):
        diff = np.where(fin, np.abs(c - r), 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(diff == 0.0, 0.0, np.where(b > 0.0, diff / b, np.inf))
    ratio = np.where(fin, ratio, np.where(same_nf, 0.0, np.inf))
    n = ratio.size
    if n == 0:
        return dict(max_ratio=0.0, median_ratio=0.0, normwise=0.0, n_fail=0, count=0)
    srt = np.sort(ratio)
    num = float(np.sqrt(np.sum(diff * diff)))
    den = float(np.sqrt(np.sum(np.where(fin, r * r, 0.0))))
    normwise = 0.0 if num == 0.0 else (num / den if den > 0.0 else float("inf"))
    return dict(max_ratio=float(srt[-1]), median_ratio=float(srt[(n - 1) // 2]),
                normwise=normwise, n_fail=int(np.count_nonzero(ratio > 1.0)), count=int(n))
