// SSYRK and STRSM on the SGEMM core (Level-3 BLAS, whose other routines are
// written over GEMM; the paper's SGEMM implements the Level-3 BLAS SGEMM
// interface, Sec. 1).
//
// SSYRK with a split algorithm runs on the tensor cores in one launch over the
// triangle's tiles (tc_syrk.cu). Otherwise (SIMT, or alpha = 0 / k = 0) and
// for STRSM, the operation recurses by halving: the off-diagonal half-size
// block of each level is one gb_sgemm call, down to diagonal leaves of at
// most 128 rows.
//   SSYRK  leaves: every diagonal block's triangle in ONE launch of a small
//          FP32 SIMT kernel (64 x 64 tiles, the tiles above or below the
//          diagonal skipped).
//   STRSM  leaves: forward/backward substitution in one kernel per leaf, the
//          leaf's op(A) block in shared memory; left side: each warp solves
//          four columns of B at once (lanes over rows), right side: four rows
//          (lanes over columns, the rows staged through shared memory).
//          Leaves depend on one another through the GEMM updates, so they
//          run in order.
// X overwrites B in STRSM after B <- alpha B. Each GEMM update is
// B_rest <- B_rest - op(A)_block * X_done (alpha = -1, beta = 1); operand
// and output blocks are disjoint parts of the same arrays.
#include <stdint.h>

#include "internal.h"

namespace gb {
namespace {

constexpr int kLeaf = 128;       // largest diagonal leaf
constexpr int kTile = 64;        // SSYRK leaf kernel tile
constexpr int kTk = 16;

// ------------------------------------------------------------- SSYRK leaves

// All diagonal blocks (size kLeaf, the last one ragged) of an n x n C:
// blockIdx.y = block, blockIdx.x = one of its three 64 x 64 tiles on or
// beside the diagonal inside the `lower` triangle. Thread (tx, ty) of the
// 16 x 16 grid owns rows tx + 16a and columns ty + 16b of the tile.
template <bool TRANS>
__global__ void __launch_bounds__(256)
syrk_diag_kernel(int64_t n, int64_t k, float alpha, const float *__restrict__ A, int64_t lda,
                 float beta, float *__restrict__ C, int64_t ldc, int lower) {
    const int t = blockIdx.x;
    const int tr = t == 0 ? 0 : (t == 2 ? 1 : (lower ? 1 : 0));
    const int tc = t == 0 ? 0 : (t == 2 ? 1 : (lower ? 0 : 1));
    const int64_t base = (int64_t)blockIdx.y * kLeaf;
    const int64_t r0 = base + tr * kTile, c0 = base + tc * kTile;
    if (r0 >= n || c0 >= n) return;
    __shared__ float As[kTk][kTile + 4];
    __shared__ float Bs[kTk][kTile + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int64_t p0 = 0; p0 < k; p0 += kTk) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + 256 * q;
            // op(A)[i, p] = A[i + p lda] ('N') or A[p + i lda] ('T'); the
            // index split follows the contiguous dimension for coalescing
            const int i = TRANS ? e / kTk : e % kTile;
            const int p = TRANS ? e % kTk : e / kTile;
            const int64_t pp = p0 + p;
            const int64_t ri = r0 + i, ci = c0 + i;
            float va = 0.f, vb = 0.f;
            if (pp < k) {
                if (ri < n) va = TRANS ? A[pp + ri * lda] : A[ri + pp * lda];
                if (ci < n) vb = TRANS ? A[pp + ci * lda] : A[ci + pp * lda];
            }
            As[p][i] = va;
            Bs[p][i] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < kTk; ++p) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[p][tx + 16 * u];
                b[u] = Bs[p][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t i = r0 + tx + 16 * u, j = c0 + ty + 16 * v;
            if (i >= n || j >= n || (lower ? i < j : i > j)) continue;
            float *p = C + i + j * ldc;
            *p = beta == 0.f ? alpha * acc[u][v] : fmaf(alpha, acc[u][v], beta * *p);
        }
}

// ------------------------------------------------------------- STRSM leaves

constexpr int kLeafCols = 4;     // columns (left) or rows (right) per warp
constexpr int kRightRows = 8 * kLeafCols;   // rows of B per CTA, right side

// Loads op(A)'s s x s leaf block at (r0, r0) into shared memory: T[j*s + i]
// (COLMAJOR) or T[i*s + j], 0 outside the triangle, 1 on a unit diagonal
// (not read), and the reciprocals of the diagonal into D[0 .. s). Each warp
// takes stored columns w, w + 8, ... of the leaf, four at a time, with its
// lanes over stored rows (coalesced; sixteen independent loads per lane in
// flight).
template <bool COLMAJOR>
__device__ __forceinline__ void load_leaf(float *T, float *D, int s, const float *__restrict__ A,
                                          int64_t lda, int64_t r0, int trans, int tlower,
                                          int unit) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = warp; b0 < s; b0 += 32) {
        float v[4][4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int bcol = b0 + 8 * g;
            const float *src = A + r0 + (r0 + bcol) * lda;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int a = lane + 32 * r;             // stored row
                const int i = trans ? bcol : a, j = trans ? a : bcol;
                const bool inside = bcol < s && a < s && (tlower ? i >= j : i <= j) &&
                                    !(unit && i == j);
                v[g][r] = inside ? src[a] : 0.f;
            }
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int bcol = b0 + 8 * g;
            if (bcol >= s) break;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int a = lane + 32 * r;
                if (a >= s) break;
                const int i = trans ? bcol : a, j = trans ? a : bcol;
                const float x = (unit && i == j) ? 1.f : v[g][r];
                T[COLMAJOR ? j * s + i : i * s + j] = x;
                if (i == j) D[i] = unit ? 1.f : 1.f / x;
            }
        }
    }
}

// op(A)_leaf X = B_leaf for the s <= 128 rows r0 .. r0+s of B. Each warp
// solves kLeafCols columns at once (independent chains for ILP); lanes hold
// rows lane + 32r. Column-oriented substitution: x_j = b_j * (1 / t_jj), then
// b_i -= t_ij x_j for the rows still to solve, j in dependency order. (The
// reciprocal, rounded once per leaf, perturbs t_jj by at most one rounding,
// as in the reference BLAS's right-side STRSM; a division per step and
// column made the leaf instruction-bound.)
__global__ void __launch_bounds__(256)
trsm_left_leaf_kernel(int s, int64_t n, const float *__restrict__ A, int64_t lda, int64_t r0,
                      int trans, int tlower, int unit, float *__restrict__ B, int64_t ldb) {
    extern __shared__ float T[];
    float *D = T + s * s;
    load_leaf<true>(T, D, s, A, lda, r0, trans, tlower, unit);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t col0 = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * kLeafCols;
    if (col0 >= n) return;
    float b[kLeafCols][4];
#pragma unroll
    for (int q = 0; q < kLeafCols; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = lane + 32 * r;
            b[q][r] = (col0 + q < n && i < s) ? B[r0 + i + (col0 + q) * ldb] : 0.f;
        }
    if (tlower) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            for (int jj = 0; jj < 32; ++jj) {
                const int j = 32 * r + jj;
                if (j >= s) break;
                const float d = D[j];
                float x[kLeafCols];
#pragma unroll
                for (int q = 0; q < kLeafCols; ++q) {
                    const float bj = __shfl_sync(0xffffffffu, b[q][r], jj);
                    x[q] = bj * d;
                    if (lane == jj) b[q][r] = x[q];
                }
#pragma unroll
                for (int rr = r; rr < 4; ++rr) {
                    const int i = lane + 32 * rr;
                    if (i > j && i < s) {
                        const float t = T[j * s + i];
#pragma unroll
                        for (int q = 0; q < kLeafCols; ++q) b[q][rr] = fmaf(-t, x[q], b[q][rr]);
                    }
                }
            }
        }
    } else {
#pragma unroll
        for (int r = 3; r >= 0; --r) {
            for (int jj = 31; jj >= 0; --jj) {
                const int j = 32 * r + jj;
                if (j >= s) continue;
                const float d = D[j];
                float x[kLeafCols];
#pragma unroll
                for (int q = 0; q < kLeafCols; ++q) {
                    const float bj = __shfl_sync(0xffffffffu, b[q][r], jj);
                    x[q] = bj * d;
                    if (lane == jj) b[q][r] = x[q];
                }
#pragma unroll
                for (int rr = 0; rr <= r; ++rr) {
                    const int i = lane + 32 * rr;
                    if (i < j) {
                        const float t = T[j * s + i];
#pragma unroll
                        for (int q = 0; q < kLeafCols; ++q) b[q][rr] = fmaf(-t, x[q], b[q][rr]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kLeafCols; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = lane + 32 * r;
            if (col0 + q < n && i < s) B[r0 + i + (col0 + q) * ldb] = b[q][r];
        }
}

// X op(A)_leaf = B_leaf for the s <= 128 columns c0 .. c0+s of B. A CTA
// takes kRightRows rows, staged through shared memory (Bs[c][row], padded)
// so that global accesses run along the rows; each warp then solves
// kLeafCols rows at once with lanes over columns c = lane + 32r.
__global__ void __launch_bounds__(256)
trsm_right_leaf_kernel(int s, int64_t m, const float *__restrict__ A, int64_t lda, int64_t c0,
                       int trans, int tlower, int unit, float *__restrict__ B, int64_t ldb) {
    extern __shared__ float T[];
    float *D = T + s * s;
    float *Bs = D + kLeaf;                            // [s][kRightRows + 1]
    constexpr int LDS = kRightRows + 1;
    const int64_t row0 = (int64_t)blockIdx.x * kRightRows;
    load_leaf<false>(T, D, s, A, lda, c0, trans, tlower, unit);
    for (int e = threadIdx.x; e < s * kRightRows; e += blockDim.x) {
        const int rl = e % kRightRows, c = e / kRightRows;
        Bs[c * LDS + rl] = row0 + rl < m ? B[row0 + rl + (c0 + c) * ldb] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int rw = (threadIdx.x >> 5) * kLeafCols;     // this warp's first row in the CTA
    float b[kLeafCols][4];
#pragma unroll
    for (int q = 0; q < kLeafCols; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int c = lane + 32 * r;
            b[q][r] = c < s ? Bs[c * LDS + rw + q] : 0.f;
        }
    if (!tlower) {          // op(A) upper: columns left to right
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            for (int ii = 0; ii < 32; ++ii) {
                const int i = 32 * r + ii;
                if (i >= s) break;
                const float d = D[i];
                float x[kLeafCols];
#pragma unroll
                for (int q = 0; q < kLeafCols; ++q) {
                    const float bi = __shfl_sync(0xffffffffu, b[q][r], ii);
                    x[q] = bi * d;
                    if (lane == ii) b[q][r] = x[q];
                }
#pragma unroll
                for (int rr = r; rr < 4; ++rr) {
                    const int c = lane + 32 * rr;
                    if (c > i && c < s) {
                        const float t = T[i * s + c];
#pragma unroll
                        for (int q = 0; q < kLeafCols; ++q) b[q][rr] = fmaf(-x[q], t, b[q][rr]);
                    }
                }
            }
        }
    } else {                // op(A) lower: columns right to left
#pragma unroll
        for (int r = 3; r >= 0; --r) {
            for (int ii = 31; ii >= 0; --ii) {
                const int i = 32 * r + ii;
                if (i >= s) continue;
                const float d = D[i];
                float x[kLeafCols];
#pragma unroll
                for (int q = 0; q < kLeafCols; ++q) {
                    const float bi = __shfl_sync(0xffffffffu, b[q][r], ii);
                    x[q] = bi * d;
                    if (lane == ii) b[q][r] = x[q];
                }
#pragma unroll
                for (int rr = 0; rr <= r; ++rr) {
                    const int c = lane + 32 * rr;
                    if (c < i) {
                        const float t = T[i * s + c];
#pragma unroll
                        for (int q = 0; q < kLeafCols; ++q) b[q][rr] = fmaf(-x[q], t, b[q][rr]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kLeafCols; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int c = lane + 32 * r;
            if (c < s) Bs[c * LDS + rw + q] = b[q][r];
        }
    __syncthreads();
    for (int e = threadIdx.x; e < s * kRightRows; e += blockDim.x) {
        const int rl = e % kRightRows, c = e / kRightRows;
        if (row0 + rl < m) B[row0 + rl + (c0 + c) * ldb] = Bs[c * LDS + rl];
    }
}

// ------------------------------------------------------------------- host

bool is_t(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }
bool is_n(char c) { return c == 'N' || c == 'n'; }
bool is_l(char c) { return c == 'L' || c == 'l'; }
bool is_u(char c) { return c == 'U' || c == 'u'; }
int64_t max1(int64_t x) { return x > 1 ? x : 1; }

int64_t split_point(int64_t nn) {
    const int64_t h = nn / 2;
    return (h + kLeaf - 1) / kLeaf * kLeaf;
}

int check_handle(gb_handle_t h) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    return dev == h->device ? GB_OK : GB_ERR_HANDLE;
}

// One GEMM of the recursion: either records its workspace need (ws_need !=
// nullptr) or runs it.
struct GemmRunner {
    gb_handle_t h;
    gb_algo_t algo;
    void *ws;
    size_t ws_bytes;
    cudaStream_t s;
    size_t *ws_need;
    int operator()(char ta, char tb, int64_t m, int64_t n, int64_t k, float alpha, const float *A,
                   int64_t lda, const float *B, int64_t ldb, float beta, float *C,
                   int64_t ldc) const {
        if (ws_need) {
            size_t w = 0;
            int rc = gb_sgemm_workspace_size(algo, ta, tb, m, n, k, &w);
            if (rc) return rc;
            if (w > *ws_need) *ws_need = w;
            return GB_OK;
        }
        return gb_sgemm(h, algo, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws,
                        ws_bytes, s);
    }
};

// Off-diagonal blocks of SSYRK over the diagonal block [r0, r0 + nn).
int syrk_rec(const GemmRunner &g, bool lower, bool trans, int64_t r0, int64_t nn, int64_t k,
             float alpha, const float *A, int64_t lda, float beta, float *C, int64_t ldc) {
    if (nn <= kLeaf) return GB_OK;
    const int64_t n1 = split_point(nn), n2 = nn - n1;
    int rc = syrk_rec(g, lower, trans, r0, n1, k, alpha, A, lda, beta, C, ldc);
    if (rc) return rc;
    rc = syrk_rec(g, lower, trans, r0 + n1, n2, k, alpha, A, lda, beta, C, ldc);
    if (rc) return rc;
    // rows of op(A): block 1 = [r0, r0 + n1), block 2 = [r0 + n1, r0 + nn)
    const float *a1 = trans ? A + r0 * lda : A + r0;
    const float *a2 = trans ? A + (r0 + n1) * lda : A + (r0 + n1);
    const char ta = trans ? 'T' : 'N', tb = trans ? 'N' : 'T';
    if (lower)   // C21 = alpha op(A)_2 op(A)_1^T + beta C21
        return g(ta, tb, n2, n1, k, alpha, a2, lda, a1, lda, beta, C + (r0 + n1) + r0 * ldc, ldc);
    return g(ta, tb, n1, n2, k, alpha, a1, lda, a2, lda, beta, C + r0 + (r0 + n1) * ldc, ldc);
}

// Split mode of the tensor-core SSYRK path, or -1 for the recursive path
// (SIMT GEMMs and the FP32 diagonal kernel; also every scale-only call).
int syrk_tc_mode(gb_algo_t algo, int64_t k, bool scale_only) {
    if (scale_only) return -1;
    return split_mode(resolve_algo(algo, k));
}

// Bytes of op(A) split and packed once (n rows, K-major), 256-byte rounded.
size_t syrk_packed_bytes(int mode, int64_t n, int64_t k) {
    const size_t per = (size_t)split_parts(mode) * (size_t)split_kpad(mode, k) *
                       (size_t)split_elem_bytes(mode);
    return (per * (size_t)n + 255) / 256 * 256;
}

int check_syrk(char uplo, char trans, int64_t n, int64_t k, int64_t lda, int64_t ldc) {
    if (!is_l(uplo) && !is_u(uplo)) return -1;
    if (!is_n(trans) && !is_t(trans)) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    if (lda < max1(is_n(trans) ? n : k)) return -7;
    if (ldc < max1(n)) return -10;
    return GB_OK;
}

// Left side: rows [r0, r0 + mm) of op(A) and B. Right side: columns.
struct TrsmCtx {
    GemmRunner g;
    bool left, tlower, trans, unit;
    int64_t m, n;
    const float *A;
    int64_t lda;
    float *B;
    int64_t ldb;
    int sm_count;
};

// op(A)[R0.., S0..] as a GEMM operand (pointer, trans flag)
inline const float *opa_block(const TrsmCtx &c, int64_t R0, int64_t S0, char *t) {
    *t = c.trans ? 'T' : 'N';
    return c.trans ? c.A + S0 + R0 * c.lda : c.A + R0 + S0 * c.lda;
}

int trsm_leaf(const TrsmCtx &c, int64_t r0, int64_t s) {
    if (c.g.ws_need) return GB_OK;
    const size_t tri = ((size_t)s * (size_t)s + kLeaf) * sizeof(float);
    if (c.left) {
        const int64_t blocks = (c.n + 8 * kLeafCols - 1) / (8 * kLeafCols);
        trsm_left_leaf_kernel<<<(unsigned)blocks, 256, tri, c.g.s>>>(
            (int)s, c.n, c.A, c.lda, r0, c.trans, c.tlower, c.unit, c.B, c.ldb);
    } else {
        const int64_t blocks = (c.m + kRightRows - 1) / kRightRows;
        const size_t smem = tri + (size_t)s * (kRightRows + 1) * sizeof(float);
        trsm_right_leaf_kernel<<<(unsigned)blocks, 256, smem, c.g.s>>>(
            (int)s, c.m, c.A, c.lda, r0, c.trans, c.tlower, c.unit, c.B, c.ldb);
    }
    return cudaGetLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int trsm_rec(const TrsmCtx &c, int64_t r0, int64_t mm) {
    if (mm <= kLeaf) return trsm_leaf(c, r0, mm);
    const int64_t m1 = split_point(mm), m2 = mm - m1;
    const int64_t a = r0, b = r0 + m1;          // first and second half
    char t;
    int rc;
    if (c.left) {
        const bool fwd = c.tlower;
        // fwd: X_1 first, then B_2 -= op(A)[2,1] X_1; else X_2 first, B_1 -= op(A)[1,2] X_2
        rc = fwd ? trsm_rec(c, a, m1) : trsm_rec(c, b, m2);
        if (rc) return rc;
        if (fwd) {
            const float *op = opa_block(c, b, a, &t);
            rc = c.g(t, 'N', m2, c.n, m1, -1.f, op, c.lda, c.B + a, c.ldb, 1.f, c.B + b, c.ldb);
        } else {
            const float *op = opa_block(c, a, b, &t);
            rc = c.g(t, 'N', m1, c.n, m2, -1.f, op, c.lda, c.B + b, c.ldb, 1.f, c.B + a, c.ldb);
        }
        if (rc) return rc;
        return fwd ? trsm_rec(c, b, m2) : trsm_rec(c, a, m1);
    }
    const bool fwd = !c.tlower;        // X op(A) = B with op(A) upper: left to right
    rc = fwd ? trsm_rec(c, a, m1) : trsm_rec(c, b, m2);
    if (rc) return rc;
    if (fwd) {   // B[:, 2] -= X[:, 1] op(A)[1, 2]
        const float *op = opa_block(c, a, b, &t);
        rc = c.g('N', t, c.m, m2, m1, -1.f, c.B + a * c.ldb, c.ldb, op, c.lda, 1.f,
                 c.B + b * c.ldb, c.ldb);
    } else {     // B[:, 1] -= X[:, 2] op(A)[2, 1]
        const float *op = opa_block(c, b, a, &t);
        rc = c.g('N', t, c.m, m1, m2, -1.f, c.B + b * c.ldb, c.ldb, op, c.lda, 1.f,
                 c.B + a * c.ldb, c.ldb);
    }
    if (rc) return rc;
    return fwd ? trsm_rec(c, b, m2) : trsm_rec(c, a, m1);
}

int check_trsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, int64_t lda,
               int64_t ldb) {
    if (!is_l(side) && !(side == 'R' || side == 'r')) return -1;
    if (!is_l(uplo) && !is_u(uplo)) return -2;
    if (!is_n(transa) && !is_t(transa)) return -3;
    if (!is_u(diag) && !is_n(diag)) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (lda < max1(is_l(side) ? m : n)) return -9;
    if (ldb < max1(m)) return -11;
    return GB_OK;
}

bool leaf_attrs_set(int dev) {
    static bool done[64] = {};
    if (dev < 0 || dev >= 64) return false;
    if (done[dev]) return true;
    const int bytes = (kLeaf * kLeaf + kLeaf) * (int)sizeof(float);
    const int rbytes = bytes + kLeaf * (kRightRows + 1) * (int)sizeof(float);
    if (cudaFuncSetAttribute(trsm_left_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes) != cudaSuccess ||
        cudaFuncSetAttribute(trsm_right_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             rbytes) != cudaSuccess)
        return false;
    done[dev] = true;
    return true;
}

TrsmCtx trsm_ctx(const GemmRunner &g, char side, char uplo, char transa, char diag, int64_t m,
                 int64_t n, const float *A, int64_t lda, float *B, int64_t ldb, int sm_count) {
    TrsmCtx c{g};
    c.left = is_l(side);
    c.trans = is_t(transa);
    c.tlower = is_l(uplo) != c.trans;
    c.unit = is_u(diag);
    c.m = m; c.n = n;
    c.A = A; c.lda = lda; c.B = B; c.ldb = ldb;
    c.sm_count = sm_count;
    return c;
}

}  // namespace
}  // namespace gb

extern "C" {

GB_API int gb_ssyrk_workspace_size(gb_algo_t algo, char uplo, char trans, int64_t n, int64_t k,
                                   size_t *bytes) {
    using namespace gb;
    int rc = check_syrk(uplo, trans, n, k, max1(is_n(trans) ? n : k), max1(n));
    if (rc) return rc;
    if (!bytes || algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_BF16X9) return GB_ERR_ARG;
    // the larger of the two paths' needs (the path also depends on alpha)
    size_t need = 0;
    GemmRunner g{nullptr, algo, nullptr, 0, nullptr, &need};
    rc = syrk_rec(g, is_l(uplo), is_t(trans), 0, n, k, 1.f, nullptr, max1(is_n(trans) ? n : k),
                  0.f, nullptr, max1(n));
    if (rc) return rc;
    const int mode = syrk_tc_mode(algo, k, n == 0 || k == 0);
    if (mode >= 0 && syrk_packed_bytes(mode, n, k) > need) need = syrk_packed_bytes(mode, n, k);
    *bytes = need;
    return GB_OK;
}

GB_API int gb_ssyrk(gb_handle_t h, gb_algo_t algo, char uplo, char trans, int64_t n, int64_t k,
                    float alpha, const float *A, int64_t lda, float beta, float *C, int64_t ldc,
                    void *workspace, size_t ws_bytes, void *stream) {
    using namespace gb;
    int rc = check_syrk(uplo, trans, n, k, lda, ldc);
    if (rc) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_BF16X9) return GB_ERR_ARG;
    rc = check_handle(h);
    if (rc) return rc;
    if (n == 0 || ((alpha == 0.f || k == 0) && beta == 1.f)) return GB_OK;
    const bool scale_only = alpha == 0.f || k == 0;
    if (!C || (!scale_only && !A)) return GB_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mode = syrk_tc_mode(algo, k, scale_only);
    if (mode >= 0) {
        // tensor cores: split/pack op(A) once, one launch over the triangle
        const size_t need = syrk_packed_bytes(mode, n, k);
        if (ws_bytes < need || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
            return GB_ERR_WORKSPACE;
        const int64_t kpad = split_kpad(mode, k);
        if (launch_split_pack(mode, is_t(trans), n, k, A, lda, workspace, kpad, n * kpad, s) !=
            cudaSuccess)
            return GB_ERR_CUDA;
        TcSyrkArgs t{};
        t.mode = mode;
        t.packed = workspace;
        t.n = n; t.k = k;
        t.alpha = alpha; t.beta = beta;
        t.C = C; t.ldc = ldc;
        t.lower = is_l(uplo);
        t.sm_count = h->sm_count;
        t.dstate = h->dstate;
        t.wait_limit = h->wait_limit;
        return launch_tc_syrk(t, s) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
    }
    size_t need = 0;
    GemmRunner probe{nullptr, algo, nullptr, 0, nullptr, &need};
    rc = syrk_rec(probe, is_l(uplo), is_t(trans), 0, n, k, alpha, A, lda, beta, C, ldc);
    if (rc) return rc;
    if (need && (ws_bytes < need || !workspace)) return GB_ERR_WORKSPACE;
    GemmRunner g{h, algo, workspace, ws_bytes, s, nullptr};
    rc = syrk_rec(g, is_l(uplo), is_t(trans), 0, n, k, alpha, A, lda, beta, C, ldc);
    if (rc) return rc;
    const int64_t kk = scale_only ? 0 : k;
    dim3 grid(3, (unsigned)((n + kLeaf - 1) / kLeaf));
    if (is_t(trans))
        syrk_diag_kernel<true><<<grid, 256, 0, s>>>(n, kk, alpha, A, lda, beta, C, ldc, is_l(uplo));
    else
        syrk_diag_kernel<false><<<grid, 256, 0, s>>>(n, kk, alpha, A, lda, beta, C, ldc, is_l(uplo));
    return cudaGetLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

GB_API int gb_strsm_workspace_size(gb_algo_t algo, char side, char uplo, char transa, char diag,
                                   int64_t m, int64_t n, size_t *bytes) {
    using namespace gb;
    int rc = check_trsm(side, uplo, transa, diag, m, n, max1(is_l(side) ? m : n), max1(m));
    if (rc) return rc;
    if (!bytes || algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_BF16X9) return GB_ERR_ARG;
    size_t need = 0;
    GemmRunner g{nullptr, algo, nullptr, 0, nullptr, &need};
    TrsmCtx c = trsm_ctx(g, side, uplo, transa, diag, m, n, nullptr, max1(is_l(side) ? m : n),
                         nullptr, max1(m), 0);
    rc = (m == 0 || n == 0) ? GB_OK : trsm_rec(c, 0, is_l(side) ? m : n);
    if (rc) return rc;
    *bytes = need;
    return GB_OK;
}

GB_API int gb_strsm(gb_handle_t h, gb_algo_t algo, char side, char uplo, char transa, char diag,
                    int64_t m, int64_t n, float alpha, const float *A, int64_t lda, float *B,
                    int64_t ldb, void *workspace, size_t ws_bytes, void *stream) {
    using namespace gb;
    int rc = check_trsm(side, uplo, transa, diag, m, n, lda, ldb);
    if (rc) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_BF16X9) return GB_ERR_ARG;
    rc = check_handle(h);
    if (rc) return rc;
    if (m == 0 || n == 0) return GB_OK;
    if (!B || (alpha != 0.f && !A)) return GB_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (alpha == 0.f) {
        return launch_scale_c(m, n, 0.f, B, ldb, s) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
    }
    size_t need = 0;
    GemmRunner probe{nullptr, algo, nullptr, 0, nullptr, &need};
    TrsmCtx pc = trsm_ctx(probe, side, uplo, transa, diag, m, n, A, lda, B, ldb, h->sm_count);
    rc = trsm_rec(pc, 0, is_l(side) ? m : n);
    if (rc) return rc;
    if (need && (ws_bytes < need || !workspace)) return GB_ERR_WORKSPACE;
    if (!leaf_attrs_set(h->device)) return GB_ERR_CUDA;
    if (alpha != 1.f && launch_scale_c(m, n, alpha, B, ldb, s) != cudaSuccess) return GB_ERR_CUDA;
    GemmRunner g{h, algo, workspace, ws_bytes, s, nullptr};
    TrsmCtx c = trsm_ctx(g, side, uplo, transa, diag, m, n, A, lda, B, ldb, h->sm_count);
    return trsm_rec(c, 0, is_l(side) ? m : n);
}

}  // extern "C"
