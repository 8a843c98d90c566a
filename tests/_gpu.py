"""Helpers for the GPU parity tests: run one problem through the C ABI and
compare it with the CPU oracle."""
import numpy as np

import oracle
import workloads as wl

ALGOS = ("simt", "tf32x3", "bf16x3", "bf16x6", "bf16x9", "fp16x3")

# Fixed relative error each algorithm adds to a product a*b by dropping the
# smallest cross terms of its split (derivation: a = h + l + e with
# |a - h| <= u_t|a| and |e| <= u_t^2|a| for a t-bit format, u_t = 2^-t; the
# dropped l*l, e*b and a*e terms are each <= u_t^2 |ab| up to (1 + u_t)^2):
#   TF32 x 2 terms (t = 11): 3 * 2^-22;  BF16 x 2 terms (t = 8): 3 * 2^-16;
#   BF16 x 3 terms: the split is exact, the dropped pairs of weight 2^-24
#   contribute 2 * 2^-24; with all nine products nothing is dropped.
#   FP16 x 2 terms on scaled rows (t = 11, as TF32): 3 * 2^-22 for every
#   element within 2^17 of its row's (op(A)) or 2^28 of its column block's
#   (op(B)) largest magnitude; smaller ones carry the absolute term of
#   fp16x3_floor.
#   Rounded up slightly for the (1 + u_t) factors.
SPLIT_EXTRA = {"simt": 0.0, "tf32x3": 3.01 * 2.0 ** -22, "bf16x3": 3.03 * 2.0 ** -16,
               "bf16x6": 2.02 * 2.0 ** -24, "bf16x9": 0.0, "fp16x3": 3.01 * 2.0 ** -22}
# The tensor cores' accumulation, under the library's model (each MMA
# instruction adds its 16 exact products, 8 for TF32, to the running sum
# with an error of at most one FP32 ulp = 2u): products per pair of terms P
# and products per instruction Q give P*ceil(K/Q) steps, so accumulation
# and the alpha/beta epilogue stay within (2*P*ceil(K/Q) + 2)*u*D; what
# that exceeds of the plain 2*max(K,1)*u*D is added to the bound.
PRODUCTS = {"tf32x3": (3, 8), "bf16x3": (3, 16), "bf16x6": (6, 16), "bf16x9": (9, 16),
            "fp16x3": (3, 16)}
# K from which the split meets the plain FP32 bound 2*K*u*D under that model
# (the dropped terms fit in what the accumulation leaves; BF16 x 2 terms
# within half of it).
STANDARD_BOUND_MIN_K = {"simt": 0, "tf32x3": 16, "bf16x3": 1024, "bf16x6": 9, "bf16x9": 10,
                        "fp16x3": 16}


def split_extra(algo, k):
    """The relative term beyond 2*max(K,1)*u of algo's own bound at this K."""
    if algo not in PRODUCTS:
        return SPLIT_EXTRA.get(algo, 0.0)
    P, Q = PRODUCTS[algo]
    k = max(int(k), 1)
    steps = P * ((k + Q - 1) // Q)
    return SPLIT_EXTRA[algo] + max(0, 2 * steps + 2 - 2 * k) * 2.0 ** -24


def auto_algo(k):
    """The algorithm AUTO runs at this K (the library's rule)."""
    return "bf16x3" if k >= 1024 else ("bf16x6" if k >= STANDARD_BOUND_MIN_K["bf16x6"] else "simt")


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


def op_arrays(p):
    """op(A) (M x K) and op(B) (K x N) of a problem as float64 arrays."""
    A = p.A[:p.m, :p.k] if p.ta == "N" else p.A[:p.k, :p.m].T
    B = p.B[:p.k, :p.n] if p.tb == "N" else p.B[:p.n, :p.k].T
    return A.astype(np.float64), B.astype(np.float64)


def fp16x3_floor(p, cols=None):
    """The absolute term of the scaled FP16 split's bound, per element (i, j):
        |alpha| 2^-34 (2^(lg a_i - 3) sum_p |b_pj| + 2^(lg b_J - 14) sum_p |a_ip|)
    with lg a_i = floor(log2 max_p |a_ip|) over row i of op(A), and lg b_J the
    same over the block of 256 columns of op(B) holding column j (finite
    entries). Derivation: a row of op(A) is scaled so that its largest
    magnitude lies in [2^3, 2^4) and an element x of it is kept as h + l 2^-11
    with h, l in FP16; each rounding to FP16 errs by at most 2^-11 of its value
    or half the subnormal spacing 2^-25, so |x - h - l 2^-11| <= 2^-22 |x| +
    2^-36 in scaled units, i.e. 2^-36 2^-e_i = 2^(lg a_i - 3 - 36) absolutely;
    likewise 2^(lg b_J - 14 - 36) for op(B) (column blocks to [2^14, 2^15)).
    Each such absolute error meets the other operand's magnitudes in the
    products; 2^-34 covers both roundings of the split and the (1 + 2^-22)
    factors with room. The relative 2^-22 parts make the 3 * 2^-22 of
    SPLIT_EXTRA."""
    A, B = op_arrays(p)
    absA = np.where(np.isfinite(A), np.abs(A), 0.0)
    absB = np.where(np.isfinite(B), np.abs(B), 0.0)

    def lg(m):
        return np.where(m > 0, np.frexp(m)[1] - 1, 0)   # floor(log2 m) for m > 0

    la = lg(absA.max(axis=1))
    colmax = absB.max(axis=0)
    blk = np.arange(p.n) // 256
    blockmax = np.zeros(blk[-1] + 1 if p.n else 0)
    np.maximum.at(blockmax, blk, colmax)
    lb = lg(blockmax[blk])
    Sa = absA.sum(axis=1)
    Sb = absB.sum(axis=0)
    if cols is not None:
        lb, Sb = lb[cols], Sb[cols]
    return abs(float(p.alpha)) * 2.0 ** -34 * (np.ldexp(1.0, la - 3)[:, None] * Sb[None, :]
                                             + np.ldexp(1.0, lb - 14)[None, :] * Sa[:, None])


def assert_within_bound(p, got, cols=None, algo="simt"):
    """The algorithm's own bound (2*max(K,1)*u + extra_algo)*D always (for the
    scaled FP16 split plus its absolute term, fp16x3_floor), and the plain
    FP32 bound 2*max(K,1)*u*D when K >= STANDARD_BOUND_MIN_K[algo] (for the
    scaled FP16 split on the elements whose absolute term is at most a
    quarter of the plain bound)."""
    C64, D = oracle_of(p, cols)
    sub = got[:p.m, :] if cols is None else got[:p.m, cols]
    std = oracle.err_report(sub, C64, D, p.k)
    if algo == "fp16x3":
        F = fp16x3_floor(p, cols)
        c = sub.astype(np.float64)
        fin = np.isfinite(c) & np.isfinite(C64)
        assert np.array_equal(fin, np.isfinite(C64)), "fp16x3: non-finite where the oracle is finite"
        diff = np.abs(c[fin] - C64[fin])
        own = oracle.bound(D[fin], p.k, split_extra(algo, p.k)) + F[fin]
        assert np.all(diff <= own), \
            f"fp16x3: {int(np.count_nonzero(diff > own))} elements over its own bound"
        if p.k >= STANDARD_BOUND_MIN_K[algo]:
            plain = oracle.bound(D[fin], p.k)
            small = F[fin] <= 0.25 * plain
            assert np.all(diff[small] <= plain[small]), "fp16x3: error over the FP32 bound"
        return std
    rep = oracle.err_report(sub, C64, D, p.k, extra=split_extra(algo, p.k))
    assert rep["max_ratio"] <= 1.0, f"{algo}: error over its own bound: {rep}"
    if p.k >= STANDARD_BOUND_MIN_K[algo]:
        assert std["max_ratio"] <= 1.0, f"{algo}: error over the FP32 bound: {std}"
    return std


def assert_bit_exact(p, got):
    C64, _ = oracle_of(p)
    want = C64.astype(np.float32)
    assert np.array_equal(got[:p.m, :], want), \
        f"not bit-exact: {np.count_nonzero(got[:p.m, :] != want)} elements differ"


def aligned_problem(ta, tb, m, n, k, alpha, beta, seed, dist="uniform"):
    """Leading dimensions padded up to a multiple of 4 (+4), so TMA can read A and B."""
    rng = np.random.default_rng(seed)
    gen = {"uniform": wl.uniform, "int": wl.int_uniform, "logu": wl.log_uniform_signed}[dist]
    ar, ac = wl.stored_shape(ta, m, k)
    br, bc = wl.stored_shape(tb, k, n)
    r4 = lambda x: (x + 3) // 4 * 4 + 4
    A = gen(rng, ar, ac, r4(ar))
    B = gen(rng, br, bc, r4(br))
    C = gen(rng, m, n, m + 3, pad=wl.CANARY)
    return wl.Problem(ta, tb, m, n, k, float(np.float32(alpha)), float(np.float32(beta)),
                      A, A.shape[0], B, B.shape[0], C, C.shape[0])
