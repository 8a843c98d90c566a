// Plain FP32 SGEMM on the CUDA cores: C <- alpha*op(A)*op(B) + beta*C,
// column-major, all four transpose combinations, any leading dimension.
//
// The paper's design (Sec. 2 and 3) keeps a 1 x 5 block of C in registers,
// reuses each loaded A value against five B columns, stages a k-block of A
// and B in L1 and streams the k dimension. The same three ideas, sized for
// an sm_103a SM:
//   * register tile: every thread owns an 8 x 8 block of C (64 FP32
//     accumulators) and, per k, reuses 8 A values against 8 B values
//     (64 FMA per 4 shared-memory vector loads);
//   * shared-memory staging: a 128 x 8 panel of op(A) and an 8 x 128 panel
//     of op(B) per CTA (256 threads), double-buffered, the next panel
//     prefetched into registers while the current one is consumed (the
//     analogue of the paper's A' prefetch);
//   * whole-K accumulation: C is read and written once, in the epilogue,
//     where alpha/beta are applied with fused multiply-adds.
// Global loads are coalesced in both storage orders: a panel whose stored
// matrix is contiguous along M (or N) is read along M; one contiguous along
// K is read along K and transposed on its way into shared memory. float4
// loads are used when every address involved is 16-byte aligned.
#include "f32x2.cuh"
#include "internal.h"

namespace gb {
namespace {

constexpr int BM = 128, BN = 128, BK = 8;
constexpr int NT = 256;
constexpr int LDS = BM + 4;   // padded shared row (floats); conflict-free transposed stores

// Loads this thread's four elements of a 128 x 8 panel of op(X), where op(X)
// is (rows x K) and the panel starts at (r0, k0). KC: the stored matrix is
// contiguous along K (element (r,p) at X[p + r*ld]); otherwise contiguous
// along the rows (element (r,p) at X[r + p*ld]). VEC: 16-byte loads allowed.
template <bool KC, bool VEC>
__device__ __forceinline__ void load_panel(const float *__restrict__ X, int64_t ld,
                                           int64_t rows, int64_t K, int64_t r0, int64_t k0,
                                           int t, float v[4]) {
    if (!KC) {
        // rows-contiguous: 32 threads cover 128 rows of one k column
        const int p = t >> 5;
        const int64_t kk = k0 + p;
        if (VEC) {
            const int r = (t & 31) * 4;
            const int64_t rr = r0 + r;
            if (kk < K && rr + 3 < rows) {
                float4 q = __ldg(reinterpret_cast<const float4 *>(X + rr + kk * ld));
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    v[e] = (kk < K && rr + e < rows) ? __ldg(X + rr + e + kk * ld) : 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t rr = r0 + (t & 31) + 32 * e;
                v[e] = (kk < K && rr < rows) ? __ldg(X + rr + kk * ld) : 0.f;
            }
        }
    } else {
        if (VEC) {
            // K-contiguous, 16-byte loads: thread -> row t/2, k-quad (t&1)*4
            const int64_t rr = r0 + (t >> 1);
            const int64_t kk = k0 + (t & 1) * 4;
            if (rr < rows && kk + 3 < K) {
                float4 q = __ldg(reinterpret_cast<const float4 *>(X + kk + rr * ld));
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    v[e] = (rr < rows && kk + e < K) ? __ldg(X + kk + e + rr * ld) : 0.f;
            }
        } else {
            // K-contiguous, scalar: 8 consecutive k of 4 rows per warp instruction
            const int64_t kk = k0 + (t & 7);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t rr = r0 + (t >> 3) + 32 * e;
                v[e] = (rr < rows && kk < K) ? __ldg(X + kk + rr * ld) : 0.f;
            }
        }
    }
}

// Stores the four elements loaded by load_panel into the [BK][LDS] panel.
template <bool KC, bool VEC>
__device__ __forceinline__ void store_panel(float *__restrict__ S, int t, const float v[4]) {
    if (!KC) {
        const int p = t >> 5;
        if (VEC) {
            *reinterpret_cast<float4 *>(S + p * LDS + (t & 31) * 4) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) S[p * LDS + (t & 31) + 32 * e] = v[e];
        }
    } else {
        if (VEC) {
            const int r = t >> 1, p = (t & 1) * 4;
#pragma unroll
            for (int e = 0; e < 4; ++e) S[(p + e) * LDS + r] = v[e];
        } else {
            const int p = t & 7;
#pragma unroll
            for (int e = 0; e < 4; ++e) S[p * LDS + (t >> 3) + 32 * e] = v[e];
        }
    }
}

template <bool TA, bool TB, bool VA, bool VB, bool VC>
__global__ void __launch_bounds__(NT, 2)
simt_sgemm_kernel(int64_t M, int64_t N, int64_t K, float alpha, float beta,
                  const float *__restrict__ A, int64_t lda,
                  const float *__restrict__ B, int64_t ldb,
                  float *__restrict__ C, int64_t ldc) {
    // op(A) is M x K: stored A is K-contiguous iff transposed.
    // op(B) is K x N; we stage op(B)^T (N x K) panels: stored B is
    // K-contiguous iff NOT transposed.
    constexpr bool AKC = TA;
    constexpr bool BKC = !TB;
    __shared__ __align__(16) float As[2][BK * LDS];
    __shared__ __align__(16) float Bs[2][BK * LDS];

    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int64_t n0 = (int64_t)blockIdx.y * BN;

    // acc2[ip][j]: rows (2ip, 2ip + 1) of the thread's 8 (tx*4 + 0..3,
    // 64 + tx*4 + 0..3), column j of its 8, as one FP32 pair
    unsigned long long acc2[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc2[i][j] = 0ull;

    const int64_t nk = (K + BK - 1) / BK;
    float ra[4], rb[4];
    if (nk > 0) {
        load_panel<AKC, VA>(A, lda, M, K, m0, 0, t, ra);
        load_panel<BKC, VB>(B, ldb, N, K, n0, 0, t, rb);
        store_panel<AKC, VA>(As[0], t, ra);
        store_panel<BKC, VB>(Bs[0], t, rb);
    }
    __syncthreads();

    int cur = 0;
    for (int64_t kt = 0; kt < nk; ++kt) {
        const bool more = kt + 1 < nk;
        if (more) {
            load_panel<AKC, VA>(A, lda, M, K, m0, (kt + 1) * BK, t, ra);
            load_panel<BKC, VB>(B, ldb, N, K, n0, (kt + 1) * BK, t, rb);
        }
        const float *as = As[cur];
        const float *bs = Bs[cur];
#pragma unroll
        for (int p = 0; p < BK; ++p) {
            // a pairs straight from two 16-byte loads; b from two 16-byte
            // loads, each value made a (b_j, b_j) pair in registers
            const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(as + p * LDS + tx * 4);
            const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(as + p * LDS + 64 + tx * 4);
            const float4 bl = *reinterpret_cast<const float4 *>(bs + p * LDS + ty * 4);
            const float4 bh = *reinterpret_cast<const float4 *>(bs + p * LDS + 64 + ty * 4);
            const unsigned long long a[4] = {a0.x, a0.y, a1.x, a1.y};
            const unsigned long long b[8] = {pack2(bl.x, bl.x), pack2(bl.y, bl.y), pack2(bl.z, bl.z),
                                             pack2(bl.w, bl.w), pack2(bh.x, bh.x), pack2(bh.y, bh.y),
                                             pack2(bh.z, bh.z), pack2(bh.w, bh.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) ffma2(acc2[i][j], a[i], b[j]);
        }
        if (more) {
            store_panel<AKC, VA>(As[cur ^ 1], t, ra);
            store_panel<BKC, VB>(Bs[cur ^ 1], t, rb);
        }
        __syncthreads();
        cur ^= 1;
    }

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) unpack2(acc2[i][j], acc[2 * i][j], acc[2 * i + 1][j]);

    // Epilogue: thread rows {tx*4 + 0..3, 64 + tx*4 + 0..3}, columns
    // {ty*4 + 0..3, 64 + ty*4 + 0..3}; a warp writes 64 consecutive floats of
    // a column per store instruction. With beta != 0 every C value of the
    // thread is read before the first store (a store may alias a later load,
    // so interleaving them would serialise the loads' latencies).
    if (beta != 0.f) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t col = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
            const float *cc = C + col * ldc;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + h * 64 + tx * 4;
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                if (col < N) {
                    if (VC && row + 3 < M) {
                        const float4 q = *reinterpret_cast<const float4 *>(cc + row);
                        c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) c[e] = row + e < M ? cc[row + e] : 0.f;
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[h * 4 + e][j] = fmaf(alpha, acc[h * 4 + e][j], beta * c[e]);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] *= alpha;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t col = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
        if (col >= N) continue;
        float *cc = C + col * ldc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t row = m0 + h * 64 + tx * 4;
            if (VC && row + 3 < M) {
                *reinterpret_cast<float4 *>(cc + row) =
                    make_float4(acc[h * 4 + 0][j], acc[h * 4 + 1][j], acc[h * 4 + 2][j], acc[h * 4 + 3][j]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (row + e < M) cc[row + e] = acc[h * 4 + e][j];
            }
        }
    }
}

__global__ void scale_c_kernel(int64_t M, int64_t N, float beta, float *__restrict__ C,
                               int64_t ldc) {
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % M, j = e / M;
        float *p = C + i + j * ldc;
        *p = beta != 0.f ? beta * *p : 0.f;
    }
}

__global__ void scaled_copy_kernel(int64_t M, int64_t N, float beta, const float *__restrict__ X,
                                   int64_t ldx, float *__restrict__ Y, int64_t ldy) {
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % M, j = e / M;
        Y[i + j * ldy] = beta != 0.f ? beta * X[i + j * ldx] : 0.f;
    }
}

template <bool TA, bool TB, bool VA, bool VB, bool VC>
cudaError_t launch_t(const SimtArgs &a, cudaStream_t s) {
    dim3 grid((unsigned)((a.m + BM - 1) / BM), (unsigned)((a.n + BN - 1) / BN));
    simt_sgemm_kernel<TA, TB, VA, VB, VC><<<grid, NT, 0, s>>>(
        a.m, a.n, a.k, a.alpha, a.beta, a.A, a.lda, a.B, a.ldb, a.C, a.ldc);
    return cudaGetLastError();
}

template <bool TA, bool TB>
cudaError_t launch_vec(const SimtArgs &a, bool va, bool vb, bool vc, cudaStream_t s) {
    // Instantiate the two most useful combinations: everything aligned, or
    // scalar everywhere; a mixed case takes the scalar kernel.
    if (va && vb && vc) return launch_t<TA, TB, true, true, true>(a, s);
    return launch_t<TA, TB, false, false, false>(a, s);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t launch_simt_sgemm(const SimtArgs &a, cudaStream_t s) {
    if ((a.m + BM - 1) / BM > 2147483647LL || (a.n + BN - 1) / BN > 65535LL)
        return cudaErrorInvalidConfiguration;
    const bool va = aligned16(a.A) && a.lda % 4 == 0;
    const bool vb = aligned16(a.B) && a.ldb % 4 == 0;
    const bool vc = aligned16(a.C) && a.ldc % 4 == 0;
    if (!a.ta && !a.tb) return launch_vec<false, false>(a, va, vb, vc, s);
    if (!a.ta && a.tb) return launch_vec<false, true>(a, va, vb, vc, s);
    if (a.ta && !a.tb) return launch_vec<true, false>(a, va, vb, vc, s);
    return launch_vec<true, true>(a, va, vb, vc, s);
}

cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float *C, int64_t ldc,
                           cudaStream_t s) {
    const int64_t total = m * n;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    scale_c_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, n, beta, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_scaled_copy(int64_t m, int64_t n, float beta, const float *X, int64_t ldx,
                               float *Y, int64_t ldy, cudaStream_t s) {
    const int64_t total = m * n;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    scaled_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, n, beta, X, ldx, Y, ldy);
    return cudaGetLastError();
}

}  // namespace gb
