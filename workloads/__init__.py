"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws numbers: it holds none of the GEMM arithmetic, and
neither the oracle nor the CUDA library imports it. Callers hand its arrays
to both sides.

Conventions
-----------
* Matrices are column-major float32, stored as Fortran-ordered numpy arrays
  of shape (ld, cols); the logical matrix is ``arr[:rows, :]`` and the rows
  ``rows..ld-1`` are padding.
* Values come from ``numpy.random.default_rng(seed)`` (PCG64, the same on
  every platform), drawn in float64 in column-major element order and
  rounded to float32 (round to nearest even). Matrices of one problem are
  drawn in the order A, B, C, then G.
* Padding rows of inputs hold NaN (so a kernel that reads them poisons its
  output); padding rows of outputs hold ``CANARY`` (so a kernel that writes
  them is caught).

The workloads mirror the paper's measurements (square sizes with a stride
larger than the row length, Sec. 4) and the workloads of the GB300 build:
the 384^3 plain case, the padded-stride sweep, the split-precision shapes
with log-uniform magnitudes, the dense-layer gradient case and the grouped
batch of 2000 uneven problems.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CANARY = np.float32(-12345.5)


def stored_shape(trans: str, rows: int, cols: int):
    """Shape (rows, cols) of the stored matrix whose op() is rows x cols."""
    return (rows, cols) if trans in "Nn" else (cols, rows)


def embed(vals: np.ndarray, ld: int, pad_value) -> np.ndarray:
    """Place a (rows, cols) matrix into a Fortran (ld, cols) float32 array."""
    rows, cols = vals.shape
    if ld < max(rows, 1):
        raise ValueError("ld smaller than rows")
    out = np.empty((ld, cols), dtype=np.float32, order="F")
    out[rows:, :] = pad_value
    out[:rows, :] = vals
    return out


def _colmajor(flat: np.ndarray, rows: int, cols: int) -> np.ndarray:
    # flat[i + j*rows] becomes element (i, j)
    return flat.reshape(cols, rows).T


def uniform(rng, rows, cols, ld=None, lo=-1.0, hi=1.0, pad=np.nan):
    v = rng.uniform(lo, hi, size=rows * cols)
    return embed(_colmajor(v, rows, cols).astype(np.float32), ld or max(rows, 1), pad)


def int_uniform(rng, rows, cols, ld=None, lo=-8, hi=8, pad=np.nan):
    v = rng.integers(lo, hi + 1, size=rows * cols).astype(np.float64)
    return embed(_colmajor(v, rows, cols).astype(np.float32), ld or max(rows, 1), pad)


def log_uniform_signed(rng, rows, cols, ld=None, e_lo=-20.0, e_hi=20.0, pad=np.nan):
    """Random sign times 2^U(e_lo, e_hi): exponents first, then signs."""
    n = rows * cols
    e = rng.uniform(e_lo, e_hi, size=n)
    s = rng.integers(0, 2, size=n)
    v = np.where(s == 1, -1.0, 1.0) * np.exp2(e)
    return embed(_colmajor(v, rows, cols).astype(np.float32), ld or max(rows, 1), pad)


def normal(rng, rows, cols, ld=None, std=1.0, pad=np.nan):
    v = rng.normal(0.0, std, size=rows * cols)
    return embed(_colmajor(v, rows, cols).astype(np.float32), ld or max(rows, 1), pad)


@dataclass
class Problem:
    """One SGEMM problem: C <- alpha*op(A)*op(B) + beta*C (host arrays)."""
    ta: str
    tb: str
    m: int
    n: int
    k: int
    alpha: float
    beta: float
    A: np.ndarray
    lda: int
    B: np.ndarray
    ldb: int
    C: np.ndarray
    ldc: int
    meta: dict = field(default_factory=dict)

    @property
    def flops(self) -> int:
        return 2 * self.m * self.n * self.k


def make_problem(ta, tb, m, n, k, alpha, beta, seed=None, rng=None, dist="uniform",
                 ld_pad=0, **dist_kw) -> Problem:
    """Draw A, B, C (in that order) for one problem."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    gen = {"uniform": uniform, "int": int_uniform, "logu": log_uniform_signed,
           "normal": normal}[dist]
    ar, ac = stored_shape(ta, m, k)
    br, bc = stored_shape(tb, k, n)
    lda, ldb, ldc = max(ar, 1) + ld_pad, max(br, 1) + ld_pad, max(m, 1) + ld_pad
    A = gen(rng, ar, ac, lda, **dist_kw)
    B = gen(rng, br, bc, ldb, **dist_kw)
    C = gen(rng, m, n, ldc, pad=CANARY, **dist_kw)
    return Problem(ta, tb, m, n, k, float(np.float32(alpha)), float(np.float32(beta)),
                   A, lda, B, ldb, C, ldc)


# ---- the named workloads -------------------------------------------------

def plain_384(integer=False) -> Problem:
    """M=N=K=384, 'N','N', ld=384, U[-1,1] (seed 0), alpha=1, beta=0.5.
    The integer variant draws from {-8..8} for the bit-exact check."""
    return make_problem("N", "N", 384, 384, 384, 1.0, 0.5, seed=0,
                        dist="int" if integer else "uniform")


SWEEP_SIZES = (16, 100, 257, 512, 1000, 1023, 2048, 4096, 8192)


def sweep_case(n: int, ta: str, tb: str) -> Problem:
    """Square n, leading dimensions = stored rows + 7, alpha=1.5, beta=-0.5,
    U[-1,1] from seed 1."""
    return make_problem(ta, tb, n, n, n, 1.5, -0.5, seed=1, ld_pad=7)


SPLIT_SHAPES = ((8192, 8192, 1024), (8192, 8192, 8192), (8192, 8192, 16384),
                (8192, 8192, 64), (64, 8192, 8192))


def split_case(m: int, n: int, k: int, seed: int = 2) -> Problem:
    """Random sign, magnitude 2^U(-20,20), alpha=1, beta=0, 'N','N'."""
    return make_problem("N", "N", m, n, k, 1.0, 0.0, seed=seed, dist="logu")


def dense_layer(batch=4096, d_in=1024, d_out=4096, seed=3):
    """Y = X W with X (batch x d_in), W (d_in x d_out) ~ N(0, 1/d_in) and the
    upstream gradient G ~ N(0,1) (batch x d_out); row-major float32 arrays."""
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0 / np.sqrt(d_in), size=(batch, d_in)).astype(np.float32)
    W = rng.normal(0.0, 1.0 / np.sqrt(d_in), size=(d_in, d_out)).astype(np.float32)
    G = rng.normal(0.0, 1.0, size=(batch, d_out)).astype(np.float32)
    return X, W, G


def grouped_problems(count=2000, seed=4, lo=8, hi=1024, with_data=True):
    """`count` problems with M, N, K each round(2^U(log2 lo, log2 hi)),
    trans flags 'N'/'T' with p=0.5, alpha and beta ~ U[-2,2], entries U[-1,1].

    Shapes and scalars are drawn first for all problems (M, N, K, ta, tb,
    alpha, beta per problem), then the matrices problem by problem."""
    rng = np.random.default_rng(seed)
    l0, l1 = np.log2(lo), np.log2(hi)
    shapes = []
    for _ in range(count):
        m, n, k = (int(np.clip(np.rint(np.exp2(rng.uniform(l0, l1))), lo, hi)) for _ in range(3))
        ta = "T" if rng.random() < 0.5 else "N"
        tb = "T" if rng.random() < 0.5 else "N"
        alpha = float(np.float32(rng.uniform(-2.0, 2.0)))
        beta = float(np.float32(rng.uniform(-2.0, 2.0)))
        shapes.append((ta, tb, m, n, k, alpha, beta))
    if not with_data:
        return shapes
    probs = []
    for (ta, tb, m, n, k, alpha, beta) in shapes:
        ar, ac = stored_shape(ta, m, k)
        br, bc = stored_shape(tb, k, n)
        A = uniform(rng, ar, ac)
        B = uniform(rng, br, bc)
        C = uniform(rng, m, n, pad=CANARY)
        probs.append(Problem(ta, tb, m, n, k, alpha, beta, A, ar, B, br, C, m))
    return probs
