/*
 * Reference oracle for C <- alpha*op(A)*op(B) + beta*C (SGEMM, Level-3 BLAS).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct CPU
 * definition that the CUDA library is checked against. Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library itself never calls it and shares no code with it.
 *
 * What it computes (paper Sec. 1: dense matrix multiplication costs 2MNK
 * flops with A: M x K and B: K x N, and the routine implements the SGEMM
 * interface of Level-3 BLAS):
 *
 *     C64[i,j] = alpha * sum_{p=0}^{K-1} op(A)[i,p] * op(B)[p,j] + beta * C[i,j]
 *     D[i,j]   = |alpha| * sum_p |op(A)[i,p]| * |op(B)[p,j]| + |beta| * |C[i,j]|
 *
 * All matrices are column-major: element (r,c) of X is X[r + c*ldX].
 * op(X) = X for trans 'N'/'n', X^T for 'T'/'t'/'C'/'c'.
 * The sum runs sequentially in p, in double precision, starting at +0.0.
 * Every float*float product is exact in double (24+24 <= 53 bits), so the
 * only error is the double accumulation, far below the FP32 bound.
 * D is the denominator of the per-element error bound used by the tests.
 *
 * Level-3 BLAS semantics: beta == 0 means C is not read (a NaN there does
 * not propagate); alpha == 0 means A and B are not read.
 *
 * `cols` (optional) selects which output columns j to compute: output column
 * q of C64/D holds column cols[q] of the result. This lets a caller check a
 * sample of a large product one column at a time. NULL means all N columns.
 *
 * Built with -O2 -ffp-contract=off (no fused multiply-add, no fast-math).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int is_n(char t) { return t == 'N' || t == 'n'; }
static int is_t(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }

/* op(A)[i,p] for column-major A. */
static inline float opA_f(char ta, const float *A, int64_t lda, int64_t i, int64_t p) {
    return is_n(ta) ? A[i + p * lda] : A[p + i * lda];
}
/* op(B)[p,j] for column-major B. */
static inline float opB_f(char tb, const float *B, int64_t ldb, int64_t p, int64_t j) {
    return is_n(tb) ? B[p + j * ldb] : B[j + p * ldb];
}
static inline double opA_d(char ta, const double *A, int64_t lda, int64_t i, int64_t p) {
    return is_n(ta) ? A[i + p * lda] : A[p + i * lda];
}
static inline double opB_d(char tb, const double *B, int64_t ldb, int64_t p, int64_t j) {
    return is_n(tb) ? B[p + j * ldb] : B[j + p * ldb];
}

/* alpha*s + beta*C[i,j] and the bound denominator; C is read only when
   beta != 0 (BLAS: beta == 0 means C need not be set on input). */
static inline void finish(double alpha, double beta, double s, double sa,
                          const float *C, int64_t ldc, int64_t i, int64_t j,
                          double *out, double *dout)
{
    double v = alpha * s;
    double d = fabs(alpha) * sa;
    if (beta != 0.0) {
        double c = (double)C[i + j * ldc];
        v += beta * c;
        d += fabs(beta) * fabs(c);
    }
    *out = v;
    if (dout) *dout = d;
}

/* Returns 0 on success, -1 on a bad transpose character, -2 on negative
   sizes, -3 when a work buffer cannot be allocated. */
int oracle_sgemm(char ta, char tb, int64_t m, int64_t n, int64_t k,
                 double alpha, const float *A, int64_t lda,
                 const float *B, int64_t ldb,
                 double beta, const float *C, int64_t ldc,
                 const int64_t *cols, int64_t ncols,
                 double *C64, int64_t ldc64, double *D, int64_t ldd,
                 int nthreads)
{
    if (!(is_n(ta) || is_t(ta)) || !(is_n(tb) || is_t(tb))) return -1;
    if (m < 0 || n < 0 || k < 0) return -2;
    int64_t nout = cols ? ncols : n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    /* One output column per iteration; within a column, element (i,j)
       accumulates its K products in order p = 0, 1, ..., K-1. When A is not
       transposed the i loop is innermost (unit stride in A); this interchange
       changes no element's summation order. */
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : err)
    for (int64_t q = 0; q < nout; ++q) {
        int64_t j = cols ? cols[q] : q;
        if (is_n(ta)) {
            double *s = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
            double *sa = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
            if (!s || !sa) {
                err = -3;
            } else {
                if (alpha != 0.0) {
                    for (int64_t p = 0; p < k; ++p) {
                        double b = (double)opB_f(tb, B, ldb, p, j);
                        for (int64_t i = 0; i < m; ++i) {
                            double a = (double)opA_f(ta, A, lda, i, p);
                            s[i] += a * b;
                            sa[i] += fabs(a) * fabs(b);
                        }
                    }
                }
                for (int64_t i = 0; i < m; ++i)
                    finish(alpha, beta, s[i], sa[i], C, ldc, i, j, C64 + i + q * ldc64,
                           D ? D + i + q * ldd : NULL);
            }
            free(s);
            free(sa);
        } else {
            for (int64_t i = 0; i < m; ++i) {
                double si = 0.0, sai = 0.0;
                if (alpha != 0.0) {
                    for (int64_t p = 0; p < k; ++p) {
                        double a = (double)opA_f(ta, A, lda, i, p);
                        double b = (double)opB_f(tb, B, ldb, p, j);
                        si += a * b;
                        sai += fabs(a) * fabs(b);
                    }
                }
                finish(alpha, beta, si, sai, C, ldc, i, j, C64 + i + q * ldc64,
                       D ? D + i + q * ldd : NULL);
            }
        }
    }
    if (err) return err;
    return 0;
}

/* The same definition on double inputs; used for the finite-difference
   check of the backward formulas. */
int oracle_dgemm(char ta, char tb, int64_t m, int64_t n, int64_t k,
                 double alpha, const double *A, int64_t lda,
                 const double *B, int64_t ldb,
                 double beta, const double *C, int64_t ldc,
                 double *Out, int64_t ldo, int nthreads)
{
    if (!(is_n(ta) || is_t(ta)) || !(is_n(tb) || is_t(tb))) return -1;
    if (m < 0 || n < 0 || k < 0) return -2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            if (alpha != 0.0)
                for (int64_t p = 0; p < k; ++p)
                    s += opA_d(ta, A, lda, i, p) * opB_d(tb, B, ldb, p, j);
            double v = alpha * s;
            if (beta != 0.0) v += beta * C[i + j * ldc];
            Out[i + j * ldo] = v;
        }
    }
    return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
