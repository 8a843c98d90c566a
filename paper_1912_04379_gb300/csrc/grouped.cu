// Grouped SGEMM: many independent problems C_i <- alpha_i*op(A_i)*op(B_i) +
// beta_i*C_i in one persistent launch.
//
// Plan (host, once): validate every problem with the same BLAS checks as
// gb_sgemm, drop quick-return problems, cut each remaining problem into
// output tiles of one tile class (128 x 128 with an 8 x 8 register tile per
// thread, or 64 x 64 with 4 x 4 for small problems), and sort all tiles by
// their work (K x tile area), largest first. Problem descriptors and the
// work list are uploaded once to device memory owned by the plan.
//
// Run (stream-ordered, no allocation, no host synchronisation, so a CUDA
// graph can capture it): reset the work counter in the caller's workspace,
// then launch one persistent kernel. Each CTA repeatedly takes the next
// tile from the sorted list with an atomic increment (largest tiles first,
// small ones fill the tail: longest-processing-time-first balancing) and
// computes it with the shared-memory staged FMA scheme of the plain SIMT
// kernel, transposes and leading dimensions read from the problem's
// descriptor.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace gb {
namespace {

struct GProblem {
    const float *A;
    const float *B;
    float *C;
    int64_t lda, ldb, ldc;
    int m, n, k;            // k = 0 when alpha == 0: A and B are not read
    float alpha, beta;
    int ta, tb;
};

struct GItem {
    int prob;
    int tm, tn;             // tile coordinates
    int cls;                // 0: 128 x 128, 1: 64 x 64
};

constexpr int NT = 256;

template <int BM, int BN, int BK, int RM>
struct TileCfg {
    // 256 threads as (BM/TM) x (BN/TN); TM = 4*RM rows and TN = 4*RN columns per thread
    static constexpr int TM = 4 * RM;
    static constexpr int TX = BM / TM;           // threads along M
    static constexpr int TY = NT / TX;           // threads along N
    static constexpr int TN = BN / TY;
    static constexpr int RN = TN / 4;
    static constexpr int LDA = BM + 4, LDB = BN + 4;
    static constexpr int A_PER = BM * BK / NT, B_PER = BN * BK / NT;
    static_assert(TX * TY == NT && TN % 4 == 0, "thread layout");
    static_assert(A_PER * NT == BM * BK && B_PER * NT == BN * BK, "load split");
};

// Scalar, bounds-checked load of this thread's share of a rows x BK panel
// of op(X)^(T) starting at (r0, k0). kc: stored X is K-contiguous.
template <int ROWS, int BK, int PER>
__device__ __forceinline__ void gload(const float *__restrict__ X, int64_t ld, bool kc, int rows,
                                      int K, int r0, int k0, int t, float v[PER]) {
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int l = t + NT * e;
        int r, p;
        if (kc) { p = l % BK; r = l / BK; }
        else    { r = l % ROWS; p = l / ROWS; }
        const int rr = r0 + r, pp = k0 + p;
        float x = 0.f;
        if (rr < rows && pp < K) x = kc ? __ldg(X + pp + (int64_t)rr * ld) : __ldg(X + rr + (int64_t)pp * ld);
        v[e] = x;
    }
}

template <int ROWS, int BK, int PER, int LD>
__device__ __forceinline__ void gstore(float *__restrict__ S, bool kc, int t, const float v[PER]) {
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int l = t + NT * e;
        int r, p;
        if (kc) { p = l % BK; r = l / BK; }
        else    { r = l % ROWS; p = l / ROWS; }
        S[p * LD + r] = v[e];
    }
}

template <int BM, int BN, int BK, int RM>
__device__ __forceinline__ void simt_tile(const GProblem &P, int tm, int tn, float *smem) {
    using T = TileCfg<BM, BN, BK, RM>;
    float *As = smem;                         // [2][BK][LDA]
    float *Bs = smem + 2 * BK * T::LDA;       // [2][BK][LDB]
    const int t = threadIdx.x;
    const int tx = t % T::TX, ty = t / T::TX;
    const int m0 = tm * BM, n0 = tn * BN;
    const bool akc = P.ta != 0;               // stored A K-contiguous iff transposed
    const bool bkc = P.tb == 0;               // stored B K-contiguous iff not transposed
    float acc[T::TM][T::TN];
#pragma unroll
    for (int i = 0; i < T::TM; ++i)
#pragma unroll
        for (int j = 0; j < T::TN; ++j) acc[i][j] = 0.f;

    const int nk = (P.k + BK - 1) / BK;
    float ra[T::A_PER], rb[T::B_PER];
    if (nk > 0) {
        gload<BM, BK, T::A_PER>(P.A, P.lda, akc, P.m, P.k, m0, 0, t, ra);
        gload<BN, BK, T::B_PER>(P.B, P.ldb, bkc, P.n, P.k, n0, 0, t, rb);
        gstore<BM, BK, T::A_PER, T::LDA>(As, akc, t, ra);
        gstore<BN, BK, T::B_PER, T::LDB>(Bs, bkc, t, rb);
    }
    __syncthreads();
    int cur = 0;
    for (int kt = 0; kt < nk; ++kt) {
        const bool more = kt + 1 < nk;
        if (more) {
            gload<BM, BK, T::A_PER>(P.A, P.lda, akc, P.m, P.k, m0, (kt + 1) * BK, t, ra);
            gload<BN, BK, T::B_PER>(P.B, P.ldb, bkc, P.n, P.k, n0, (kt + 1) * BK, t, rb);
        }
        const float *as = As + cur * BK * T::LDA;
        const float *bs = Bs + cur * BK * T::LDB;
#pragma unroll
        for (int p = 0; p < BK; ++p) {
            float a[T::TM], b[T::TN];
#pragma unroll
            for (int h = 0; h < RM; ++h) {
                const float4 q = *reinterpret_cast<const float4 *>(as + p * T::LDA + h * (BM / RM) + tx * 4);
                a[h * 4 + 0] = q.x; a[h * 4 + 1] = q.y; a[h * 4 + 2] = q.z; a[h * 4 + 3] = q.w;
            }
#pragma unroll
            for (int h = 0; h < T::RN; ++h) {
                const float4 q = *reinterpret_cast<const float4 *>(bs + p * T::LDB + h * (BN / T::RN) + ty * 4);
                b[h * 4 + 0] = q.x; b[h * 4 + 1] = q.y; b[h * 4 + 2] = q.z; b[h * 4 + 3] = q.w;
            }
#pragma unroll
            for (int i = 0; i < T::TM; ++i)
#pragma unroll
                for (int j = 0; j < T::TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            gstore<BM, BK, T::A_PER, T::LDA>(As + (cur ^ 1) * BK * T::LDA, akc, t, ra);
            gstore<BN, BK, T::B_PER, T::LDB>(Bs + (cur ^ 1) * BK * T::LDB, bkc, t, rb);
        }
        __syncthreads();
        cur ^= 1;
    }
#pragma unroll
    for (int j = 0; j < T::TN; ++j) {
        const int col = n0 + (j / 4) * (BN / T::RN) + ty * 4 + (j % 4);
        if (col >= P.n) continue;
        float *cc = P.C + (int64_t)col * P.ldc;
#pragma unroll
        for (int i = 0; i < T::TM; ++i) {
            const int row = m0 + (i / 4) * (BM / RM) + tx * 4 + (i % 4);
            if (row < P.m)
                cc[row] = P.beta != 0.f ? fmaf(P.alpha, acc[i][j], P.beta * cc[row])
                                        : P.alpha * acc[i][j];
        }
    }
    __syncthreads();    // shared memory is reused by the next tile
}

using Big = TileCfg<128, 128, 8, 2>;
using Small = TileCfg<64, 64, 16, 1>;
constexpr int SMEM_FLOATS_BIG = 2 * 8 * Big::LDA + 2 * 8 * Big::LDB;
constexpr int SMEM_FLOATS_SMALL = 2 * 16 * Small::LDA + 2 * 16 * Small::LDB;
constexpr int SMEM_FLOATS = SMEM_FLOATS_BIG > SMEM_FLOATS_SMALL ? SMEM_FLOATS_BIG : SMEM_FLOATS_SMALL;

__global__ void __launch_bounds__(NT, 2)
grouped_simt_kernel(const GProblem *__restrict__ probs, const GItem *__restrict__ items,
                    int nitems, int *__restrict__ counter) {
    __shared__ __align__(16) float smem[SMEM_FLOATS];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const GItem w = items[it];
        const GProblem P = probs[w.prob];
        if (w.cls == 0) simt_tile<128, 128, 8, 2>(P, w.tm, w.tn, smem);
        else            simt_tile<64, 64, 16, 1>(P, w.tm, w.tn, smem);
    }
}

bool trans_ok(char t) {
    return t == 'N' || t == 'n' || t == 'T' || t == 't' || t == 'C' || t == 'c';
}
bool is_trans(char t) { return t != 'N' && t != 'n'; }
int64_t max1(int64_t x) { return x > 1 ? x : 1; }

int check_problem(const gb_gemm_problem_t &p) {
    if (!trans_ok(p.transa)) return -1;
    if (!trans_ok(p.transb)) return -2;
    if (p.m < 0) return -3;
    if (p.n < 0) return -4;
    if (p.k < 0) return -5;
    if (p.lda < max1(is_trans(p.transa) ? p.k : p.m)) return -8;
    if (p.ldb < max1(is_trans(p.transb) ? p.n : p.k)) return -10;
    if (p.ldc < max1(p.m)) return -13;
    // The tile coordinates and per-problem sizes are 32-bit on the device.
    if (p.m > (1 << 30) || p.n > (1 << 30) || p.k > (1 << 30)) return GB_ERR_UNSUPPORTED;
    return 0;
}

}  // namespace
}  // namespace gb

struct gb_grouped_plan_s {
    int magic;
    gb_handle_t h;
    int device;
    int64_t count;
    int nitems;
    int grid;
    gb::GProblem *d_probs;
    gb::GItem *d_items;
};

namespace {
constexpr int kPlanMagic = 0x47525031;
}

extern "C" {

GB_API int gb_sgemm_grouped_plan(gb_handle_t h, gb_algo_t algo, int64_t count,
                                 const gb_gemm_problem_t *hp, gb_grouped_plan_t *plan,
                                 size_t *ws_bytes, int64_t *bad_index) {
    using namespace gb;
    if (plan) *plan = nullptr;
    if (bad_index) *bad_index = -1;
    if (!plan || !ws_bytes || count < 0 || (count > 0 && !hp)) return GB_ERR_ARG;
    if (algo != GB_ALGO_AUTO && algo != GB_ALGO_SIMT) return GB_ERR_UNSUPPORTED;
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != h->device) return GB_ERR_HANDLE;
    if (count > (int64_t)1 << 30) return GB_ERR_UNSUPPORTED;

    std::vector<GProblem> probs;
    std::vector<GItem> items;
    std::vector<double> work;
    probs.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const gb_gemm_problem_t &p = hp[i];
        int rc = check_problem(p);
        if (rc) {
            if (bad_index) *bad_index = i;
            return rc;
        }
        const bool scale_only = p.alpha == 0.f || p.k == 0;
        if (p.m == 0 || p.n == 0 || (scale_only && p.beta == 1.f)) continue;
        if (!p.C || (!scale_only && (!p.A || !p.B))) {
            if (bad_index) *bad_index = i;
            return GB_ERR_ARG;
        }
        GProblem g;
        g.A = p.A; g.B = p.B; g.C = p.C;
        g.lda = p.lda; g.ldb = p.ldb; g.ldc = p.ldc;
        g.m = (int)p.m; g.n = (int)p.n; g.k = scale_only ? 0 : (int)p.k;
        g.alpha = p.alpha; g.beta = p.beta;
        g.ta = is_trans(p.transa); g.tb = is_trans(p.transb);
        const int pi = (int)probs.size();
        probs.push_back(g);
        // Tile class: 64 x 64 when either output side is below 96 (a 128-wide
        // tile would be mostly empty), else 128 x 128.
        const int cls = (p.m < 96 || p.n < 96) ? 1 : 0;
        const int bm = cls ? 64 : 128, bn = cls ? 64 : 128;
        const int tiles_m = (int)((p.m + bm - 1) / bm), tiles_n = (int)((p.n + bn - 1) / bn);
        for (int tm = 0; tm < tiles_m; ++tm)
            for (int tn = 0; tn < tiles_n; ++tn) {
                items.push_back(GItem{pi, tm, tn, cls});
                work.push_back((double)(g.k + 8) * bm * bn);
            }
    }
    // Longest processing time first.
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<GItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    if (sorted.size() > (size_t)1 << 30) return GB_ERR_UNSUPPORTED;

    gb_grouped_plan_s *pl = new (std::nothrow) gb_grouped_plan_s();
    if (!pl) return GB_ERR_ARG;
    pl->magic = kPlanMagic;
    pl->h = h;
    pl->device = dev;
    pl->count = count;
    pl->nitems = (int)sorted.size();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_simt_kernel, NT, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    pl->grid = std::max(1, std::min(h->sm_count * per_sm, pl->nitems));
    pl->d_probs = nullptr;
    pl->d_items = nullptr;
    bool ok = true;
    if (!probs.empty())
        ok = cudaMalloc(&pl->d_probs, probs.size() * sizeof(GProblem)) == cudaSuccess &&
             cudaMemcpy(pl->d_probs, probs.data(), probs.size() * sizeof(GProblem),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !sorted.empty())
        ok = cudaMalloc(&pl->d_items, sorted.size() * sizeof(GItem)) == cudaSuccess &&
             cudaMemcpy(pl->d_items, sorted.data(), sorted.size() * sizeof(GItem),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaFree(pl->d_probs);
        cudaFree(pl->d_items);
        delete pl;
        return GB_ERR_CUDA;
    }
    *ws_bytes = 256;         // the work counter
    *plan = pl;
    return GB_OK;
}

GB_API int gb_sgemm_grouped_run(gb_grouped_plan_t plan, void *workspace, size_t ws_bytes,
                                void *stream) {
    using namespace gb;
    if (!plan || plan->magic != kPlanMagic) return GB_ERR_PLAN;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != plan->device) return GB_ERR_HANDLE;
    if (plan->nitems == 0) return GB_OK;
    if (!workspace || ws_bytes < 256 || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return GB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *counter = static_cast<int *>(workspace);
    if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess) return GB_ERR_CUDA;
    grouped_simt_kernel<<<plan->grid, NT, 0, s>>>(plan->d_probs, plan->d_items, plan->nitems,
                                                  counter);
    return cudaGetLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

GB_API int gb_sgemm_grouped_destroy(gb_grouped_plan_t plan) {
    if (!plan) return GB_OK;
    if (plan->magic != kPlanMagic) return GB_ERR_PLAN;
    cudaDeviceSynchronize();
    cudaFree(plan->d_probs);
    cudaFree(plan->d_items);
    plan->magic = 0;
    delete plan;
    return GB_OK;
}

}  // extern "C"
