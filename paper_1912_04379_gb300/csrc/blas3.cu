// SSYRK and STRSM on the SGEMM core (Level-3 BLAS, whose other routines are
// written over GEMM; the paper's SGEMM implements the Level-3 BLAS SGEMM
// interface, Sec. 1).
//
// SSYRK with a split algorithm runs on the tensor cores in one launch over the
// triangle's tiles (tc_syrk.cu). Otherwise (SIMT, or alpha = 0 / k = 0) and
// for STRSM, the operation recurses by halving: the off-diagonal half-size
// block of each level is one gb_sgemm call, down to diagonal leaves of at
// most 128 (SSYRK) or 256 (STRSM) rows.
//   SSYRK  leaves: every diagonal block's triangle in ONE launch of a small
//          FP32 SIMT kernel (64 x 64 tiles, the tiles above or below the
//          diagonal skipped).
//   STRSM  leaves: substitution in one kernel per leaf, the leaf's triangle
//          in shared memory; 64 columns (left) or rows (right) of B per CTA,
//          two per lane, each warp owning 16 rows of the solve and taking
//          the earlier warps' solved rows as named barriers release them.
//          Leaves depend on one another through the GEMM updates, so they
//          run in order.
// X overwrites B in STRSM after B <- alpha B. Each GEMM update is
// B_rest <- B_rest - op(A)_block * X_done (alpha = -1, beta = 1); operand
// and output blocks are disjoint parts of the same arrays.
#include <stdint.h>

#include <new>

#include "internal.h"
#include "f32x2.cuh"
#include "split_common.cuh"

namespace gb {
namespace {

constexpr int kLeaf = 128;       // largest SSYRK diagonal leaf
constexpr int kTLeaf = 256;      // largest STRSM diagonal leaf
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

// A leaf solves M x = b for every vector of B, with M the s x s diagonal
// block (s <= 256) of op(A) (left side; the vectors are the columns of B) or
// of op(A)^T (right side, X op(A) = B read as op(A)^T x = b; the vectors are
// the rows of B). It is put in forward lower form L' x' = b': L' = M and
// x' = x when M is lower, else L'(i, j) = M(s-1-i, s-1-j) and x'_i = x_{s-1-i}.
// Then x'_i = (b'_i - sum over j < i of L'(i, j) x'_j) / L'(i, i), i ascending.
//
// A CTA holds 64 vectors (two per lane) and sixteen warps; warp q owns rows
// [16q, 16q + 16) of every vector in registers. It subtracts the products of
// each earlier row block p as soon as warp p has solved it (p ascending,
// columns ascending within a block, so every x'_i accumulates its terms in
// j order), then solves its own 16 x 16 diagonal block. Solved blocks pass
// from warp to warp through shared memory, released by named barriers (warp
// p arrives on barrier p + 1, the warps after it wait on it). Only entries
// with j < i are ever multiplied, so a non-finite b'_j reaches exactly the
// x'_i that depend on it. A 256-row leaf does in one launch what two 128-row
// leaves and the K = 128 GEMM update between them would do.
//
// L' in shared memory keeps only the 136 16 x 16 blocks (q, p), p <= q, of
// its lower triangle, block after block in row-block order ((0,0), (1,0),
// (1,1), (2,0), ...), each column-major: -L'(i, j) at lpos(i, j), negated so
// that every subtraction is one fused multiply-add and pairs of them one
// paired FMA. Warp q reads block (q, p) as 16 columns of 16 contiguous floats.
constexpr int kBlk = 16;                        // rows per warp block
constexpr int kLeafWarps = kTLeaf / kBlk;       // 16
constexpr int kLeafThreads = 32 * kLeafWarps;   // 512
constexpr int kVecs = 64;                       // vectors per CTA (two per lane)
constexpr int kVecsPerLane = kVecs / 32;
constexpr int kHalfLeaf = kTLeaf / 2;           // 128
constexpr int kXS = kTLeaf + 4;                 // stride of each vector
constexpr int kSFloats = kLeafWarps * (kLeafWarps + 1) / 2 * kBlk * kBlk;   // 34,816
constexpr int kPrepFloats = kSFloats + kTLeaf;                              // L' and D
constexpr size_t kPrepBytes = (size_t)kPrepFloats * sizeof(float);         // 140,288
constexpr int kRawStride = kHalfLeaf + 1;                                   // prep's staging tile
constexpr int kPrepThreads = 256;

__host__ __device__ constexpr int lblock(int q, int p) { return (q * (q + 1) / 2 + p) * kBlk * kBlk; }
__host__ __device__ constexpr int lpos(int i, int j) {
    return lblock(i / kBlk, j / kBlk) + (j % kBlk) * kBlk + i % kBlk;
}
static_assert(lpos(kTLeaf - 1, kTLeaf - 1) + 1 == kSFloats, "L' layout");
static_assert(kPrepBytes % 16 == 0, "L' and D are copied in 16-byte pieces");

__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Builds every leaf's L' and D once per call into prep[b * kPrepFloats ..]
// (leaf b = rows [256 b, 256 b + s) of op(A)'s diagonal): -L'(i, j) at
// lpos(i, j) for j < i < s and 0 elsewhere in the stored blocks, then D[i] = 1 / L'(i, i) (1
// for a unit diagonal and for padding rows). One CTA per leaf and 128 x 128
// region of L' (blockIdx.y: rows/columns 0-127, rows 128-255 x columns
// 0-127, rows/columns 128-255). The stored (sr, sc) is M(sr, sc), or M(sc, sr)
// when exactly one of (right side, transposed op) holds; L'(i, j) is M(i, j),
// or M(s-1-i, s-1-j) when M is upper. The stored tile under the region is
// read (its triangle only) coalesced into shared memory, then written out in
// L' order, also coalesced.
template <bool LEFT>
__global__ void __launch_bounds__(kPrepThreads)
trsm_leaf_prep_kernel(int64_t ms, const float *__restrict__ A, int64_t lda, int trans,
                      int tlower, int unit, float *__restrict__ prep) {
    extern __shared__ float R[];                  // R[scl * kRawStride + srl]
    const int64_t r0 = (int64_t)blockIdx.x * kTLeaf;
    const int s = (int)(ms - r0 < kTLeaf ? ms - r0 : kTLeaf);
    const int ib = blockIdx.y > 0, jb = blockIdx.y > 1;
    const int i0 = kHalfLeaf * ib, j0 = kHalfLeaf * jb;
    const bool rev = LEFT ? tlower == 0 : tlower != 0;
    const bool swap = LEFT == (trans != 0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the region's M rows and columns start at mi0, mj0 (negative or past s
    // for a ragged leaf: those are skipped); stored ones at sr0, sc0
    const int mi0 = rev ? s - i0 - kHalfLeaf : i0, mj0 = rev ? s - j0 - kHalfLeaf : j0;
    const int sr0 = swap ? mj0 : mi0, sc0 = swap ? mi0 : mj0;
    for (int scl = warp; scl < kHalfLeaf; scl += kPrepThreads / 32) {
        const int sc = sc0 + scl;
#pragma unroll
        for (int k = 0; k < kHalfLeaf / 32; ++k) {
            const int srl = lane + 32 * k, sr = sr0 + srl;
            if (sr < 0 || sr >= s || sc < 0 || sc >= s) continue;
            const int mi = swap ? sc : sr, mj = swap ? sr : sc;
            const int i = rev ? s - 1 - mi : mi, j = rev ? s - 1 - mj : mj;
            if (i > j || (i == j && !unit))
                R[scl * kRawStride + srl] = A[(r0 + sr) + (r0 + sc) * lda];
        }
    }
    __syncthreads();
    float *out = prep + (int64_t)blockIdx.x * kPrepFloats;
    for (int e = tid; e < kHalfLeaf * kHalfLeaf; e += kPrepThreads) {
        const int i = i0 + (e & (kHalfLeaf - 1)), j = j0 + e / kHalfLeaf;
        if (j / kBlk > i / kBlk) continue;         // above the diagonal blocks: not stored
        float v = 0.f;
        if (i < s && j < i) {
            const int mi = rev ? s - 1 - i : i, mj = rev ? s - 1 - j : j;
            const int sr = swap ? mj : mi, sc = swap ? mi : mj;
            v = -R[(sc - sc0) * kRawStride + (sr - sr0)];
        }
        out[lpos(i, j)] = v;
    }
    if (ib == jb && tid < kHalfLeaf) {
        const int i = i0 + tid;
        float d = 1.f;
        if (i < s && !unit) {
            const int mi = rev ? s - 1 - i : i;
            d = 1.f / R[(mi - sc0) * kRawStride + (mi - sr0)];
        }
        out[kSFloats + i] = d;
    }
}

// The leaf at rows (left) or columns (right) [r0, r0 + s) of B, its L' and D
// prepared in prep (kPrepFloats, 16-byte aligned).
// With xp non-null the solved rows (left) or columns (right) are also
// split into their three BF16 terms and stored into the packed copy of X:
// term p of vector v, position r0 + i at xp[p * xps + v * xkpad + r0 + i]
// (the layout of a packed GEMM operand whose K index is the row (left) or
// column (right) of X), so that the updates read X without a pack pass.
template <bool LEFT>
__global__ void __launch_bounds__(kLeafThreads, 1)
trsm_leaf_kernel(int s, int64_t nvec, int64_t r0, int tlower, const float *__restrict__ prep,
                 float *__restrict__ B, int64_t ldb, __nv_bfloat16 *__restrict__ xp,
                 int64_t xkpad, int64_t xps) {
    extern __shared__ __align__(16) float smem[];
    float *S = smem;                      // -L', at lpos(i, j)
    float *D = S + kSFloats;              // D[i] = 1 / L'(i, i)
    float *X = D + kTLeaf;                // X[v * kXS + i] = x'_i of vector v, once solved
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const bool rev = LEFT ? tlower == 0 : tlower != 0;    // M upper
    const int64_t v0 = (int64_t)blockIdx.x * kVecs;
    const int nblk = (s + kBlk - 1) / kBlk;
    if (q >= nblk) return;                // the named barriers count only warps < nblk

    // Every warp loads what it alone reads, so none waits for a CTA-wide
    // load phase: its row of L' blocks ((q, 0) .. (q, q), contiguous), its 16
    // reciprocals, and rows [16q, 16q + 16) of its lane's two vectors.
    {
        const int b = lblock(q, 0), nchunk = (q + 1) * kBlk * kBlk / 4;
        for (int k = lane; k < nchunk; k += 32) cp_async16(S + b + 4 * k, prep + b + 4 * k);
        if (lane < kBlk / 4) cp_async16(D + q * kBlk + 4 * lane, prep + kSFloats + q * kBlk + 4 * lane);
    }
    const int i0 = q * kBlk;                          // leaf rows i0 .. i0 + 15
    const int nv = s - i0 < kBlk ? s - i0 : kBlk;     // of which valid
    const int b0 = rev ? s - i0 - kBlk : i0;          // stored rows b0 .. b0 + 15 (reversed when rev)
    const bool full = nv == kBlk;
    const bool bvec = LEFT && full && !(reinterpret_cast<uintptr_t>(B) & 15) && ldb % 4 == 0 &&
                      (r0 + b0) % 4 == 0;
    float x[kVecsPerLane][kBlk];                      // x[h][r]: leaf row i0 + r of vector lane + 32h
    if (LEFT) {
        // coalesced: half a warp per vector (16 rows = 64 contiguous bytes),
        // staged through this warp's own rows of X, which nothing else
        // touches before this warp has solved them
        const int r = lane & (kBlk - 1);
        const int64_t brow = r0 + (rev ? s - 1 - (i0 + r) : i0 + r);
        float *xs = X + i0 + r;
        float t[kVecs / 2];
#pragma unroll
        for (int k = 0; k < kVecs / 2; ++k) {
            const int64_t v = v0 + 2 * k + (lane >> 4);
            t[k] = (r < nv && v < nvec) ? B[brow + v * ldb] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kVecs / 2; ++k) xs[(2 * k + (lane >> 4)) * kXS] = t[k];
        __syncwarp();
#pragma unroll
        for (int h = 0; h < kVecsPerLane; ++h) {
            const float4 *xq = reinterpret_cast<const float4 *>(X + (lane + 32 * h) * kXS + i0);
#pragma unroll
            for (int g = 0; g < kBlk / 4; ++g) {
                const float4 f = xq[g];
                x[h][4 * g] = f.x; x[h][4 * g + 1] = f.y; x[h][4 * g + 2] = f.z; x[h][4 * g + 3] = f.w;
            }
        }
    } else {
        const float *bb = B + (v0 + lane) + r0 * ldb;
        const int64_t vl = nvec - (v0 + lane);        // vector lane + 32h exists iff 32h < vl
#pragma unroll
        for (int r = 0; r < kBlk; ++r) {
            const int col = rev ? s - 1 - (i0 + r) : i0 + r;
#pragma unroll
            for (int h = 0; h < kVecsPerLane; ++h)
                x[h][r] = (r < nv && 32 * h < vl) ? bb[32 * h + col * ldb] : 0.f;
        }
    }
    cp_async_wait_all();
    __syncwarp();

    // xx[h][r]: rows (2r, 2r + 1) of x[h] as one FP32 pair; each pair of rows
    // takes one paired FMA per term
    unsigned long long xx[kVecsPerLane][kBlk / 2];
#pragma unroll
    for (int h = 0; h < kVecsPerLane; ++h)
#pragma unroll
        for (int r = 0; r < kBlk / 2; ++r) xx[h][r] = pack2(x[h][2 * r], x[h][2 * r + 1]);
#pragma unroll 1
    for (int p = 0; p < q; ++p) {
        named_bar_sync(1 + p, 32 * (nblk - p));       // block p solved
        const float *sp = S + lblock(q, p);           // block (q, p), column-major
#pragma unroll
        for (int cg = 0; cg < kBlk / 4; ++cg) {
            float4 yv[kVecsPerLane];                  // x'_j of columns 4cg .. 4cg + 3 of block p
#pragma unroll
            for (int h = 0; h < kVecsPerLane; ++h)
                yv[h] = *reinterpret_cast<const float4 *>(X + (lane + 32 * h) * kXS + p * kBlk + 4 * cg);
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                const ulonglong2 *lc = reinterpret_cast<const ulonglong2 *>(sp + (4 * cg + c4) * kBlk);
                unsigned long long yy[kVecsPerLane];
#pragma unroll
                for (int h = 0; h < kVecsPerLane; ++h) {
                    const float y = c4 == 0 ? yv[h].x : c4 == 1 ? yv[h].y : c4 == 2 ? yv[h].z : yv[h].w;
                    yy[h] = pack2(y, y);
                }
#pragma unroll
                for (int g = 0; g < kBlk / 4; ++g) {
                    const ulonglong2 l = lc[g];            // -L' of rows 4g .. 4g + 3
#pragma unroll
                    for (int h = 0; h < kVecsPerLane; ++h) {
                        ffma2(xx[h][2 * g], l.x, yy[h]);
                        ffma2(xx[h][2 * g + 1], l.y, yy[h]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < kVecsPerLane; ++h)
#pragma unroll
        for (int r = 0; r < kBlk / 2; ++r) unpack2(xx[h][r], x[h][2 * r], x[h][2 * r + 1]);
    {
        float d[kBlk];
        const float4 *dq = reinterpret_cast<const float4 *>(D + q * kBlk);
#pragma unroll
        for (int g = 0; g < kBlk / 4; ++g) {
            const float4 f = dq[g];
            d[4 * g] = f.x; d[4 * g + 1] = f.y; d[4 * g + 2] = f.z; d[4 * g + 3] = f.w;
        }
        const float *sq = S + lblock(q, q);
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {                  // the diagonal block, column by column
#pragma unroll
            for (int h = 0; h < kVecsPerLane; ++h) x[h][j] *= d[j];
            const float4 *lc = reinterpret_cast<const float4 *>(sq + j * kBlk);
#pragma unroll
            for (int g = (j + 1) / 4; g < kBlk / 4; ++g) {
                const float4 l = lc[g];
                const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * g + e > j)
#pragma unroll
                        for (int h = 0; h < kVecsPerLane; ++h)
                            x[h][4 * g + e] = fmaf(lv[e], x[h][j], x[h][4 * g + e]);
            }
        }
    }
    if (q + 1 < nblk) {                               // the later warps read this block
#pragma unroll
        for (int h = 0; h < kVecsPerLane; ++h) {
            float4 *xo = reinterpret_cast<float4 *>(X + (lane + 32 * h) * kXS + q * kBlk);
#pragma unroll
            for (int g = 0; g < kBlk / 4; ++g)
                xo[g] = make_float4(x[h][4 * g], x[h][4 * g + 1], x[h][4 * g + 2], x[h][4 * g + 3]);
        }
        named_bar_arrive(1 + q, 32 * (nblk - q));
    }

    // The solved rows go out while the later warps are still solving.
    if (LEFT) {
#pragma unroll
        for (int h = 0; h < kVecsPerLane; ++h) {
            const int64_t v = v0 + lane + 32 * h;
            if (v >= nvec) continue;
            float *bp = B + r0 + v * ldb;
            if (bvec) {
#pragma unroll
                for (int g = 0; g < kBlk / 4; ++g) {
                    float t[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        t[e] = rev ? x[h][kBlk - 1 - (4 * g + e)] : x[h][4 * g + e];
                    *reinterpret_cast<float4 *>(bp + b0 + 4 * g) = make_float4(t[0], t[1], t[2], t[3]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < kBlk; ++r)
                    if (r < nv) bp[rev ? s - 1 - (i0 + r) : i0 + r] = x[h][r];
            }
        }
    } else {
        float *bb = B + (v0 + lane) + r0 * ldb;
        const int64_t vl = nvec - (v0 + lane);
#pragma unroll
        for (int r = 0; r < kBlk; ++r) {
            if (r >= nv) break;
            const int col = rev ? s - 1 - (i0 + r) : i0 + r;
#pragma unroll
            for (int h = 0; h < kVecsPerLane; ++h)
                if (32 * h < vl) bb[32 * h + col * ldb] = x[h][r];
        }
    }
    if (xp) {
        const bool xvec = full && !(reinterpret_cast<uintptr_t>(xp) & 15) && xkpad % 8 == 0 &&
                          xps % 8 == 0 && (r0 + b0) % 8 == 0;
#pragma unroll
        for (int h = 0; h < kVecsPerLane; ++h) {
            const int64_t v = v0 + lane + 32 * h;
            if (v >= nvec) continue;
            __nv_bfloat16 *xv = xp + v * xkpad + r0;
            unsigned short tb[3][kBlk];                   // terms' bits, leaf row order
#pragma unroll
            for (int r = 0; r < kBlk; ++r) {
                __nv_bfloat16 t[3];
                split_bf16<3>(x[h][r], t);
#pragma unroll
                for (int p = 0; p < 3; ++p) tb[p][r] = __bfloat16_as_ushort(t[p]);
            }
            if (xvec) {
                // positions b0 .. b0 + 15, two 16-byte stores per term
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        unsigned w[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int t0 = 8 * half + 2 * k, t1 = t0 + 1;
                            const unsigned lo = rev ? tb[p][kBlk - 1 - t0] : tb[p][t0];
                            const unsigned hi = rev ? tb[p][kBlk - 1 - t1] : tb[p][t1];
                            w[k] = lo | (hi << 16);
                        }
                        *reinterpret_cast<uint4 *>(xv + p * xps + b0 + 8 * half) =
                            make_uint4(w[0], w[1], w[2], w[3]);
                    }
            } else {
#pragma unroll
                for (int r = 0; r < kBlk; ++r) {
                    if (r >= nv) break;
                    const int pos = rev ? s - 1 - (i0 + r) : i0 + r;
#pragma unroll
                    for (int p = 0; p < 3; ++p) xv[p * xps + pos] = __ushort_as_bfloat16(tb[p][r]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------- host

// Shared memory of a leaf CTA: L' (kSFloats), the diagonal reciprocals
// (256) and the 64 vectors' solved rows (kXS floats each): 206,848 bytes.
size_t leaf_smem_bytes() {
    return (size_t)(kSFloats + kTLeaf + kVecs * kXS) * sizeof(float);
}

// Shared memory of a prep CTA: one stored 128 x 128 tile, padded.
size_t prep_smem_bytes() { return (size_t)kHalfLeaf * kRawStride * sizeof(float); }

// STRSM workspace: the GEMM updates' area first (256-byte rounded), then
// every leaf's prepared L' and D.
// STRSM workspace: the GEMM updates' area first (256-byte rounded), then
// every leaf's prepared L' and D, then (pack-once updates) op(A) and X in
// split form: three BF16 terms each, rows of kpad = split_kpad(BF16 x 3, ms)
// elements, ms rows for op(A) and vecs rows (columns of B on the left, rows
// on the right) for X.
struct TrsmWorkspace {
    size_t gemm_bytes, prep_offset, ap_offset, xp_offset, total;
    int64_t kpad;
};
TrsmWorkspace trsm_workspace(size_t gemm_need, int64_t ms, int64_t vecs, bool pack_once) {
    TrsmWorkspace w;
    w.gemm_bytes = gemm_need;
    w.prep_offset = (gemm_need + 255) / 256 * 256;
    size_t off = w.prep_offset + (size_t)((ms + kTLeaf - 1) / kTLeaf) * kPrepBytes;
    w.kpad = pack_once ? split_kpad(2, ms) : 0;
    w.ap_offset = (off + 255) / 256 * 256;
    if (pack_once) off = w.ap_offset + 3 * (size_t)ms * (size_t)w.kpad * 2;
    w.xp_offset = (off + 255) / 256 * 256;
    if (pack_once) off = w.xp_offset + 3 * (size_t)vecs * (size_t)w.kpad * 2;
    w.total = off;
    return w;
}

// Pack-once updates for the BF16 splits (AUTO among them: its updates are
// BF16 x 2 or x 3 terms except for K < 9, which keep their own gb_sgemm).
bool trsm_pack_once(gb_algo_t algo) {
    return algo == GB_ALGO_AUTO || algo == GB_ALGO_SPLIT_BF16X3 || algo == GB_ALGO_SPLIT_BF16X6 ||
           algo == GB_ALGO_SPLIT_BF16X9;
}

bool is_t(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }
bool is_n(char c) { return c == 'N' || c == 'n'; }
bool is_l(char c) { return c == 'L' || c == 'l'; }
bool is_u(char c) { return c == 'U' || c == 'u'; }
int64_t max1(int64_t x) { return x > 1 ? x : 1; }

// STRSM's split: every leaf starts at a multiple of 256 rows.
int64_t trsm_split_point(int64_t nn) {
    const int64_t h = nn / 2;
    return (h + kTLeaf - 1) / kTLeaf * kTLeaf;
}

// SSYRK's split: every diagonal leaf starts at a multiple of 128 rows.
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
    const int mode = split_mode(resolve_algo(algo, k));
    return mode == 4 ? 0 : mode;   // no triangle kernel for the scaled FP16 split: TF32X3
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
    const float *prep;      // every leaf's L' and D (kPrepFloats per 256 rows)
    // Pack-once updates (BF16 splits): op(A) split and packed once (ap: as
    // the updates' op(A) on the left, as their op(B) on the right), and X
    // in the same split form, written by the leaves (xp); both rows of
    // xkpad elements, three terms. Null: each update is one gb_sgemm.
    bool pack_once = false;
    const __nv_bfloat16 *ap = nullptr;
    __nv_bfloat16 *xp = nullptr;
    int64_t xkpad = 0;
};

// One update, C -= op(A)_gemm op(B)_gemm with K = kk. With pack-once updates
// and a BF16 split for this K: a compute launch on views of the packed op(A)
// (rows a_row0.. on the left; as op(B), columns b_row0.. on the right) and
// the packed X, K range [k0, k0 + kk). Otherwise one gb_sgemm (or, when
// probing, its workspace need).
int trsm_gemm(const TrsmCtx &c, char ta, char tb, int64_t M, int64_t N, int64_t kk,
              const float *A, int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc,
              int64_t a_row0, int64_t b_row0, int64_t k0) {
    if (c.pack_once) {
        const int mode = split_mode(resolve_algo(c.g.algo, kk));
        if (mode >= 1 && mode <= 3) {
            if (c.g.ws_need) return GB_OK;
            const int64_t ms = c.left ? c.m : c.n, vecs = c.left ? c.n : c.m;
            const void *Ap = c.left ? (const void *)c.ap : (const void *)c.xp;
            const void *Bp = c.left ? (const void *)c.xp : (const void *)c.ap;
            return compute_packed_view(c.g.h, mode, M, N, kk, -1.f, Ap, c.left ? ms : vecs, a_row0,
                                       Bp, c.left ? vecs : ms, b_row0, 1.f, C, ldc, c.g.s, k0,
                                       c.xkpad);
        }
    }
    return c.g(ta, tb, M, N, kk, -1.f, A, lda, B, ldb, 1.f, C, ldc);
}

// op(A)[R0.., S0..] as a GEMM operand (pointer, trans flag)
inline const float *opa_block(const TrsmCtx &c, int64_t R0, int64_t S0, char *t) {
    *t = c.trans ? 'T' : 'N';
    return c.trans ? c.A + S0 + R0 * c.lda : c.A + R0 + S0 * c.lda;
}

int trsm_leaf(const TrsmCtx &c, int64_t r0, int64_t s) {
    if (c.g.ws_need) return GB_OK;
    const size_t smem = leaf_smem_bytes();
    const int64_t vecs = c.left ? c.n : c.m;
    const int64_t blocks = (vecs + kVecs - 1) / kVecs;
    const float *prep = c.prep + (r0 / kTLeaf) * kPrepFloats;
    if (c.left)
        trsm_leaf_kernel<true><<<(unsigned)blocks, kLeafThreads, smem, c.g.s>>>(
            (int)s, c.n, r0, c.tlower, prep, c.B, c.ldb, c.xp, c.xkpad, vecs * c.xkpad);
    else
        trsm_leaf_kernel<false><<<(unsigned)blocks, kLeafThreads, smem, c.g.s>>>(
            (int)s, c.m, r0, c.tlower, prep, c.B, c.ldb, c.xp, c.xkpad, vecs * c.xkpad);
    return cudaGetLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int trsm_rec(const TrsmCtx &c, int64_t r0, int64_t mm) {
    if (mm <= kTLeaf) return trsm_leaf(c, r0, mm);
    const int64_t m1 = trsm_split_point(mm), m2 = mm - m1;
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
            rc = trsm_gemm(c, t, 'N', m2, c.n, m1, op, c.lda, c.B + a, c.ldb, c.B + b, c.ldb,
                           b, 0, a);
        } else {
            const float *op = opa_block(c, a, b, &t);
            rc = trsm_gemm(c, t, 'N', m1, c.n, m2, op, c.lda, c.B + b, c.ldb, c.B + a, c.ldb,
                           a, 0, b);
        }
        if (rc) return rc;
        return fwd ? trsm_rec(c, b, m2) : trsm_rec(c, a, m1);
    }
    const bool fwd = !c.tlower;        // X op(A) = B with op(A) upper: left to right
    rc = fwd ? trsm_rec(c, a, m1) : trsm_rec(c, b, m2);
    if (rc) return rc;
    if (fwd) {   // B[:, 2] -= X[:, 1] op(A)[1, 2]
        const float *op = opa_block(c, a, b, &t);
        rc = trsm_gemm(c, 'N', t, c.m, m2, m1, c.B + a * c.ldb, c.ldb, op, c.lda,
                       c.B + b * c.ldb, c.ldb, 0, b, a);
    } else {     // B[:, 1] -= X[:, 2] op(A)[2, 1]
        const float *op = opa_block(c, b, a, &t);
        rc = trsm_gemm(c, 'N', t, c.m, m1, m2, c.B + b * c.ldb, c.ldb, op, c.lda,
                       c.B + a * c.ldb, c.ldb, 0, a, b);
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
    const int bytes = (int)leaf_smem_bytes(), prep_bytes = (int)prep_smem_bytes();
    if (cudaFuncSetAttribute(trsm_leaf_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes) != cudaSuccess ||
        cudaFuncSetAttribute(trsm_leaf_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes) != cudaSuccess ||
        cudaFuncSetAttribute(trsm_leaf_prep_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             prep_bytes) != cudaSuccess ||
        cudaFuncSetAttribute(trsm_leaf_prep_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             prep_bytes) != cudaSuccess)
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
    if (!bytes || algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
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
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
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
    if (!bytes || algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    size_t need = 0;
    GemmRunner g{nullptr, algo, nullptr, 0, nullptr, &need};
    TrsmCtx c = trsm_ctx(g, side, uplo, transa, diag, m, n, nullptr, max1(is_l(side) ? m : n),
                         nullptr, max1(m), 0);
    if (m == 0 || n == 0) {
        *bytes = 0;
        return GB_OK;
    }
    c.pack_once = trsm_pack_once(algo);
    rc = trsm_rec(c, 0, is_l(side) ? m : n);
    if (rc) return rc;
    *bytes = trsm_workspace(need, is_l(side) ? m : n, is_l(side) ? n : m, c.pack_once).total;
    return GB_OK;
}

}  // extern "C"

namespace gb {
namespace {

// The whole of one STRSM call after its checks, enqueued on s.
int strsm_run(gb_handle_t h, gb_algo_t algo, char side, char uplo, char transa, char diag,
              int64_t m, int64_t n, float alpha, const float *A, int64_t lda, float *B,
              int64_t ldb, void *workspace, const TrsmWorkspace &w, bool pack_once,
              cudaStream_t s) {
    const int64_t ms = is_l(side) ? m : n;
    if (alpha != 1.f && launch_scale_c(m, n, alpha, B, ldb, s) != cudaSuccess) return GB_ERR_CUDA;
    GemmRunner g{h, algo, workspace, w.gemm_bytes, s, nullptr};
    TrsmCtx c = trsm_ctx(g, side, uplo, transa, diag, m, n, A, lda, B, ldb, h->sm_count);
    float *prep = reinterpret_cast<float *>(static_cast<char *>(workspace) + w.prep_offset);
    c.prep = prep;
    const dim3 prep_grid((unsigned)((ms + kTLeaf - 1) / kTLeaf), 3);
    if (c.left)
        trsm_leaf_prep_kernel<true><<<prep_grid, kPrepThreads, prep_smem_bytes(), s>>>(
            ms, A, lda, c.trans, c.tlower, c.unit, prep);
    else
        trsm_leaf_prep_kernel<false><<<prep_grid, kPrepThreads, prep_smem_bytes(), s>>>(
            ms, A, lda, c.trans, c.tlower, c.unit, prep);
    if (cudaGetLastError() != cudaSuccess) return GB_ERR_CUDA;
    if (pack_once) {
        // op(A) split once: as the updates' op(A) (left) or op(B) (right);
        // the leaves then write X in the same form
        char *ws = static_cast<char *>(workspace);
        c.pack_once = true;
        c.ap = reinterpret_cast<const __nv_bfloat16 *>(ws + w.ap_offset);
        c.xp = reinterpret_cast<__nv_bfloat16 *>(ws + w.xp_offset);
        c.xkpad = w.kpad;
        if (pack_operand_rows(2, c.left, c.trans, ms, ms, A, lda, ws + w.ap_offset, ms, 0, s) !=
            cudaSuccess)
            return GB_ERR_CUDA;
    }
    return trsm_rec(c, 0, ms);
}

// One STRSM call's arguments and settings, and its launches captured as an
// instantiated graph: a call with the same arguments (and handle settings)
// replays the graph instead of issuing its ~70 dependent launches again.
struct TrsmGraph {
    bool valid = false;
    gb_algo_t algo{};
    char side = 0, uplo = 0, transa = 0, diag = 0;
    int64_t m = 0, n = 0, lda = 0, ldb = 0;
    float alpha = 0.f;
    const float *A = nullptr;
    float *B = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t promote_k = 0, wait_limit = 0;
    int rb_override = 0, n_gemm_rb = 0;
    bool skinny = false, fused = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;      // the stream the launches are captured on
};

bool same_call(const TrsmGraph &G, gb_handle_t h, gb_algo_t algo, char side, char uplo,
               char transa, char diag, int64_t m, int64_t n, float alpha, const float *A,
               int64_t lda, float *B, int64_t ldb, void *ws, size_t ws_bytes) {
    return G.valid && G.algo == algo && G.side == side && G.uplo == uplo && G.transa == transa &&
           G.diag == diag && G.m == m && G.n == n && G.alpha == alpha && G.A == A &&
           G.lda == lda && G.B == B && G.ldb == ldb && G.ws == ws && G.ws_bytes == ws_bytes &&
           G.promote_k == h->promote_k && G.wait_limit == h->wait_limit &&
           G.rb_override == h->rb_override && G.n_gemm_rb == h->n_gemm_rb &&
           G.skinny == h->skinny_split && G.fused == h->fused_split;
}

}  // namespace

void destroy_trsm_graph(gb_handle_t h) {
    TrsmGraph *G = static_cast<TrsmGraph *>(h->trsm_graph);
    if (!G) return;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->cs) cudaStreamDestroy(G->cs);
    delete G;
    h->trsm_graph = nullptr;
}

}  // namespace gb

extern "C" {

GB_API int gb_strsm(gb_handle_t h, gb_algo_t algo, char side, char uplo, char transa, char diag,
                    int64_t m, int64_t n, float alpha, const float *A, int64_t lda, float *B,
                    int64_t ldb, void *workspace, size_t ws_bytes, void *stream) {
    using namespace gb;
    int rc = check_trsm(side, uplo, transa, diag, m, n, lda, ldb);
    if (rc) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
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
    pc.pack_once = trsm_pack_once(algo);
    const int64_t ms = is_l(side) ? m : n, vecs = is_l(side) ? n : m;
    rc = trsm_rec(pc, 0, ms);
    if (rc) return rc;
    const TrsmWorkspace w = trsm_workspace(need, ms, vecs, pc.pack_once);
    if (ws_bytes < w.total || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 15))
        return GB_ERR_WORKSPACE;
    if (!leaf_attrs_set(h->device)) return GB_ERR_CUDA;
    // Inside the caller's own stream capture: enqueue the launches there.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return GB_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone)
        return strsm_run(h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace,
                         w, pc.pack_once, s);
    // Otherwise replay the cached graph of an identical call, or capture
    // this one (on the handle's own stream) and keep it.
    if (!h->trsm_graph) h->trsm_graph = new (std::nothrow) TrsmGraph();
    TrsmGraph *G = static_cast<TrsmGraph *>(h->trsm_graph);
    if (!G)
        return strsm_run(h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace,
                         w, pc.pack_once, s);
    if (same_call(*G, h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace,
                  ws_bytes))
        return cudaGraphLaunch(G->exec, s) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
    G->valid = false;
    if (!G->cs && cudaStreamCreateWithFlags(&G->cs, cudaStreamNonBlocking) != cudaSuccess) {
        G->cs = nullptr;
        return strsm_run(h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace,
                         w, pc.pack_once, s);
    }
    if (cudaStreamBeginCapture(G->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return strsm_run(h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace,
                         w, pc.pack_once, s);
    }
    rc = strsm_run(h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace, w,
                   pc.pack_once, G->cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(G->cs, &graph);
    cudaGraphExec_t exec = nullptr;
    const bool ok = rc == GB_OK && ec == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        // nothing ran: enqueue the call directly (it reports its own errors)
        cudaGetLastError();                 // a failed capture leaves no sticky error
        if (exec) cudaGraphExecDestroy(exec);
        return strsm_run(h, algo, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, workspace,
                         w, pc.pack_once, s);
    }
    if (G->exec) cudaGraphExecDestroy(G->exec);
    G->exec = exec;
    G->valid = true;
    G->algo = algo; G->side = side; G->uplo = uplo; G->transa = transa; G->diag = diag;
    G->m = m; G->n = n; G->alpha = alpha; G->A = A; G->lda = lda; G->B = B; G->ldb = ldb;
    G->ws = workspace; G->ws_bytes = ws_bytes;
    G->promote_k = h->promote_k; G->wait_limit = h->wait_limit;
    G->rb_override = h->rb_override; G->n_gemm_rb = h->n_gemm_rb;
    G->skinny = h->skinny_split; G->fused = h->fused_split;
    return cudaGraphLaunch(G->exec, s) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

}  // extern "C"
