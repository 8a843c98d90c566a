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
#include <math.h>
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
    // beta != 0: read every C value of this thread before the first store (a
    // store may alias a later load, so interleaving them would serialise the
    // loads' latencies), folding beta*C into the accumulators.
    if (P.beta != 0.f) {
#pragma unroll
        for (int j = 0; j < T::TN; ++j) {
            const int col = n0 + (j / 4) * (BN / T::RN) + ty * 4 + (j % 4);
            const float *cc = P.C + (int64_t)col * P.ldc;
#pragma unroll
            for (int i = 0; i < T::TM; ++i) {
                const int row = m0 + (i / 4) * (BM / RM) + tx * 4 + (i % 4);
                const float c = (row < P.m && col < P.n) ? cc[row] : 0.f;
                acc[i][j] = fmaf(P.alpha, acc[i][j], P.beta * c);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < T::TM; ++i)
#pragma unroll
            for (int j = 0; j < T::TN; ++j) acc[i][j] *= P.alpha;
    }
#pragma unroll
    for (int j = 0; j < T::TN; ++j) {
        const int col = n0 + (j / 4) * (BN / T::RN) + ty * 4 + (j % 4);
        if (col >= P.n) continue;
        float *cc = P.C + (int64_t)col * P.ldc;
#pragma unroll
        for (int i = 0; i < T::TM; ++i) {
            const int row = m0 + (i / 4) * (BM / RM) + tx * 4 + (i % 4);
            if (row < P.m) cc[row] = acc[i][j];
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
    int grid;
    // SIMT part
    int nitems;
    gb::GProblem *d_probs;
    gb::GItem *d_items;
    // tensor-core part: packed operands, tensor maps, problems, tiles and
    // pack tiles, all in device memory owned by the plan. Tiles are grouped
    // by (split mode, kernel configuration): one launch per segment present,
    // segment mode * kGroupedConfigVariants + configuration, LPT order within.
    int64_t tc_nitems, tc_npack;
    int64_t tc_seg_off[4 * gb::kGroupedConfigVariants], tc_seg_n[4 * gb::kGroupedConfigVariants];
    void *tc_packed;
    CUtensorMap *tc_maps;
    gb::TcProblem *tc_probs;
    gb::TcItem *tc_items;
    gb::PackItem *tc_pack;
};

namespace {

constexpr int kPlanMagic = 0x47525031;
constexpr int kClasses = 8;
constexpr int kPrefAuto = -1;

// Split mode of one tensor-core problem (K >= kMinKBf16x6): the preferred
// mode when it meets the FP32 bound 2*K*u*D at this K (TF32 x 2 terms from
// K >= 16, BF16 x 2 terms from K >= 1024, all 9 BF16 products from K >= 10),
// else BF16 x 3 terms with 6 products, which holds from K >= 9. AUTO takes
// the cheapest mode that holds: BF16 x 2 terms at K >= 1024, else BF16 x 3
// terms.
int tc_mode_for(int pref, int64_t k) {
    switch (pref) {
        case 0: return k >= 16 ? 0 : 2;
        case 2: return 2;
        case 3: return k >= gb::kMinKBf16x9 ? 3 : 2;
        default: return k >= 1024 ? 1 : 2;   // kPrefAuto and BF16 x 2 terms
    }
}

// Size class of a problem: floor(log2 of the geometric mean of M, N, K),
// clamped to [3, 10] and shifted to 0..7.
int size_class(int64_t m, int64_t n, int64_t k) {
    const double g = cbrt((double)m * (double)n * (double)(k > 0 ? k : 1));
    int c = (int)floor(log2(g > 1.0 ? g : 1.0)) - 3;
    return c < 0 ? 0 : (c >= kClasses ? kClasses - 1 : c);
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void free_plan_memory(gb_grouped_plan_s *pl) {
    cudaFree(pl->d_probs);
    cudaFree(pl->d_items);
    cudaFree(pl->tc_packed);
    cudaFree(pl->tc_maps);
    cudaFree(pl->tc_probs);
    cudaFree(pl->tc_items);
    cudaFree(pl->tc_pack);
}

template <class T>
bool upload(T **dptr, const std::vector<T> &v) {
    *dptr = nullptr;
    if (v.empty()) return true;
    return cudaMalloc(dptr, v.size() * sizeof(T)) == cudaSuccess &&
           cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Routing values of a size class: 0 = SIMT 64 x 64 tiles, 1 = SIMT 128 x 128
// tiles, 2 + v = tensor cores in grouped configuration v.
constexpr int kChoices = 2 + gb::kGroupedConfigVariants;

// Builds a plan for validated problems; choice[c] routes size class c.
// Returns a GB status; on error frees everything it allocated.
// pref: preferred split mode of the tensor-core problems (kPrefAuto: by K).
int build_plan(gb_handle_t h, int dev, const std::vector<gb_gemm_problem_t> &ps,
               const int choice[kClasses], int pref, gb_grouped_plan_s **out) {
    using namespace gb;
    std::vector<GProblem> probs;
    std::vector<GItem> items;
    std::vector<double> work;
    struct TcPending { size_t prob; size_t off_a, off_b; int mode, v; };
    std::vector<TcPending> tcs;
    size_t packed_bytes = 0;
    auto route_choice = [&](const gb_gemm_problem_t &p, bool scale_only) {
        return (scale_only || p.k < gb::kMinKBf16x6) ? (p.m < 96 || p.n < 96 ? 0 : 1)
                                       : choice[size_class(p.m, p.n, p.k)];
    };
    // 0 / 1: SIMT tiles, 2: tensor cores (configuration route_choice - 2)
    auto route = [&](const gb_gemm_problem_t &p, bool scale_only) {
        const int c = route_choice(p, scale_only);
        return c >= 2 ? 2 : c;
    };
    // Under AUTO, the BF16 x 2 terms problems (K >= 1024) get a launch of
    // their own only if they fill at least one round of the persistent grid;
    // fewer tiles join the BF16 x 3 terms launch (which meets the bound too),
    // since a nearly empty extra launch costs more than the extra products.
    bool x2_own_launch = true;
    if (pref == kPrefAuto) {
        int64_t x2_tiles = 0;
        for (const gb_gemm_problem_t &p : ps) {
            const bool so = p.alpha == 0.f || p.k == 0;
            if (p.m == 0 || p.n == 0 || so || route(p, so) != 2 || tc_mode_for(pref, p.k) != 1)
                continue;
            const int64_t bn1 = tc_grouped_tile_n(route_choice(p, so) - 2);
            x2_tiles += ((p.m + 127) / 128) * ((p.n + bn1 - 1) / bn1);
        }
        x2_own_launch = x2_tiles >= 2 * h->sm_count;   // one round: two CTAs per SM
    }
    for (size_t i = 0; i < ps.size(); ++i) {
        const gb_gemm_problem_t &p = ps[i];
        const bool scale_only = p.alpha == 0.f || p.k == 0;
        if (p.m == 0 || p.n == 0 || (scale_only && p.beta == 1.f)) continue;
        const int ch = route(p, scale_only);
        if (ch == 2) {
            int mode = tc_mode_for(pref, p.k);
            if (mode == 1 && !x2_own_launch) mode = 2;
            const size_t kpad = (size_t)split_kpad(mode, p.k);
            const size_t per = (size_t)split_parts(mode) * kpad * (size_t)split_elem_bytes(mode);
            TcPending t{i, packed_bytes, 0, mode, route_choice(p, scale_only) - 2};
            packed_bytes += round_up(per * (size_t)p.m, 1024);
            t.off_b = packed_bytes;
            packed_bytes += round_up(per * (size_t)p.n, 1024);
            tcs.push_back(t);
            continue;
        }
        GProblem g;
        g.A = p.A; g.B = p.B; g.C = p.C;
        g.lda = p.lda; g.ldb = p.ldb; g.ldc = p.ldc;
        g.m = (int)p.m; g.n = (int)p.n; g.k = scale_only ? 0 : (int)p.k;
        g.alpha = p.alpha; g.beta = p.beta;
        g.ta = is_trans(p.transa); g.tb = is_trans(p.transb);
        const int pi = (int)probs.size();
        probs.push_back(g);
        const int cls = ch == 1 ? 0 : 1;                 // GItem class 0: 128 x 128, 1: 64 x 64
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
    pl->count = (int64_t)ps.size();
    pl->nitems = (int)sorted.size();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_simt_kernel, NT, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    pl->grid = std::max(1, std::min(h->sm_count * per_sm, std::max(pl->nitems, 1)));
    bool ok = upload(&pl->d_probs, probs) && upload(&pl->d_items, sorted);

    // ---- tensor-core problems: packed buffers, tensor maps, tiles, pack tiles
    if (ok && !tcs.empty()) {
        ok = cudaMalloc(&pl->tc_packed, packed_bytes) == cudaSuccess &&
             cudaMalloc(&pl->tc_maps, 2 * tcs.size() * sizeof(CUtensorMap)) == cudaSuccess;
        std::vector<CUtensorMap> maps(2 * tcs.size());
        std::vector<TcProblem> tprobs(tcs.size());
        std::vector<TcItem> titems;
        std::vector<double> twork;
        std::vector<int> tmode;
        std::vector<PackItem> pack;
        char *base = static_cast<char *>(pl->tc_packed);
        for (size_t j = 0; ok && j < tcs.size(); ++j) {
            const gb_gemm_problem_t &p = ps[tcs[j].prob];
            const int mode = tcs[j].mode, v = tcs[j].v;
            const int bn = tc_grouped_tile_n(v);
            const int64_t kpad = split_kpad(mode, p.k);
            char *pa = base + tcs[j].off_a, *pb = base + tcs[j].off_b;
            ok = tc_make_grouped_operand_map(&maps[2 * j], mode, v, pa, p.k, p.m, true) &&
                 tc_make_grouped_operand_map(&maps[2 * j + 1], mode, v, pb, p.k, p.n, false);
            TcProblem &t = tprobs[j];
            t.mapA = pl->tc_maps + 2 * j;
            t.mapB = pl->tc_maps + 2 * j + 1;
            t.C = p.C; t.ldc = p.ldc;
            t.m = p.m; t.n = p.n; t.k = p.k;
            t.alpha = p.alpha; t.beta = p.beta;
            const int tiles_m = (int)((p.m + 127) / 128), tiles_n = (int)((p.n + bn - 1) / bn);
            for (int tm = 0; tm < tiles_m; ++tm)
                for (int tn = 0; tn < tiles_n; ++tn) {
                    titems.push_back(TcItem{(int)j, tm, tn, 0});
                    twork.push_back((double)p.k * bn);
                    tmode.push_back(mode * kGroupedConfigVariants + v);   // segment
                }
            // pack tiles of op(A) (M x K, K-contiguous iff A is transposed) and
            // op(B)^T (N x K, K-contiguous iff B is not transposed)
            for (int side = 0; side < 2; ++side) {
                PackItem it{};
                it.X = side ? p.B : p.A;
                it.ld = side ? p.ldb : p.lda;
                it.out = side ? pb : pa;
                it.kpad = kpad;
                it.rows = side ? p.n : p.m;
                it.ps = it.rows * kpad;
                it.k = p.k;
                it.kc = side ? !is_trans(p.transb) : is_trans(p.transa);
                it.mode = mode;
                it.vec = ((reinterpret_cast<uintptr_t>(it.X) & 15) == 0) && (it.ld % 4 == 0);
                for (int64_t r0 = 0; r0 < it.rows; r0 += 64)
                    for (int64_t p0 = 0; p0 < kpad; p0 += 64) {
                        it.r0 = r0;
                        it.p0 = p0;
                        pack.push_back(it);
                    }
            }
        }
        std::vector<int> tord(titems.size());
        for (size_t i = 0; i < tord.size(); ++i) tord[i] = (int)i;
        std::stable_sort(tord.begin(), tord.end(), [&](int a, int b) {
            return tmode[a] != tmode[b] ? tmode[a] < tmode[b] : twork[a] > twork[b];
        });
        std::vector<TcItem> tsorted(titems.size());
        for (size_t i = 0; i < tord.size(); ++i) {
            tsorted[i] = titems[tord[i]];
            ++pl->tc_seg_n[tmode[tord[i]]];
        }
        for (int sg = 1; sg < 4 * kGroupedConfigVariants; ++sg)
            pl->tc_seg_off[sg] = pl->tc_seg_off[sg - 1] + pl->tc_seg_n[sg - 1];
        ok = ok &&
             cudaMemcpy(pl->tc_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             upload(&pl->tc_probs, tprobs) && upload(&pl->tc_items, tsorted) &&
             upload(&pl->tc_pack, pack);
        pl->tc_nitems = (int64_t)tsorted.size();
        pl->tc_npack = (int64_t)pack.size();
    }
    if (!ok) {
        free_plan_memory(pl);
        delete pl;
        return GB_ERR_CUDA;
    }
    *out = pl;
    return GB_OK;
}

// A plan with both parts runs them at once: the SIMT part on the handle's
// side stream (forked from `s` before the tensor-core launches, joined back
// after), one persistent SIMT CTA per SM beside each persistent tensor-core
// CTA (together 62 K of the 64 K registers), so the SIMT tiles use the issue
// slots the latency-bound small tensor-core tiles leave idle (2000-problem
// group, AUTO: 1.00 -> 0.94 ms). Fork and join are events, so a run stays
// capturable in a CUDA graph.
int run_plan(gb_grouped_plan_s *plan, void *workspace, cudaStream_t s) {
    using namespace gb;
    gb_handle_t h = plan->h;
    const bool both = plan->tc_nitems > 0 && plan->nitems > 0 && h->side_ready;
    if (both && (cudaEventRecord(h->side_event[0], s) != cudaSuccess ||
                 cudaStreamWaitEvent(h->side_stream, h->side_event[0], 0) != cudaSuccess))
        return GB_ERR_CUDA;
    if (plan->tc_nitems > 0) {
        if (launch_split_pack_grouped(plan->tc_pack, plan->tc_npack, s) != cudaSuccess)
            return GB_ERR_CUDA;
        for (int sg = 0; sg < 4 * kGroupedConfigVariants; ++sg) {
            if (plan->tc_seg_n[sg] == 0) continue;
            if (launch_tc_grouped(sg / kGroupedConfigVariants, sg % kGroupedConfigVariants,
                                  plan->tc_probs, plan->tc_items + plan->tc_seg_off[sg],
                                  plan->tc_seg_n[sg], plan->h->sm_count, plan->h->dstate,
                                  plan->h->wait_limit, s) != cudaSuccess)
                return GB_ERR_CUDA;
        }
    }
    if (plan->nitems > 0) {
        cudaStream_t ss = both ? h->side_stream : s;
        int *counter = static_cast<int *>(workspace);
        if (cudaMemsetAsync(counter, 0, sizeof(int), ss) != cudaSuccess) return GB_ERR_CUDA;
        const int grid = both ? std::min(plan->grid, h->sm_count) : plan->grid;
        grouped_simt_kernel<<<grid, NT, 0, ss>>>(plan->d_probs, plan->d_items, plan->nitems,
                                                 counter);
        if (cudaGetLastError() != cudaSuccess) return GB_ERR_CUDA;
        if (both && (cudaEventRecord(h->side_event[1], ss) != cudaSuccess ||
                     cudaStreamWaitEvent(s, h->side_event[1], 0) != cudaSuccess))
            return GB_ERR_CUDA;
    }
    return GB_OK;
}

}  // namespace

void gb::destroy_side(gb_handle_t h) {
    if (!h->side_ready) return;
    cudaStreamDestroy(h->side_stream);
    cudaEventDestroy(h->side_event[0]);
    cudaEventDestroy(h->side_event[1]);
    h->side_ready = false;
}

namespace {

// The side stream and fork/join events of plans with both parts, created
// once per handle.
bool ensure_side(gb_handle_t h) {
    if (h->side_ready) return true;
    if (cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->side_event[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->side_event[1], cudaEventDisableTiming) != cudaSuccess)
        return false;
    h->side_ready = true;
    return true;
}

void destroy_plan(gb_grouped_plan_s *plan) {
    cudaDeviceSynchronize();
    free_plan_memory(plan);
    plan->magic = 0;
    delete plan;
}

// Synthetic square problems of side d over one buffer (A, B, C per problem).
std::vector<gb_gemm_problem_t> synthetic(float *buf, int64_t g, int64_t d, int64_t first) {
    const size_t per = (size_t)(3 * d * d);
    std::vector<gb_gemm_problem_t> ps((size_t)g);
    for (int64_t i = 0; i < g; ++i) {
        gb_gemm_problem_t &p = ps[(size_t)i];
        p.transa = ((first + i) & 1) ? 'T' : 'N';
        p.transb = ((first + i) & 2) ? 'T' : 'N';
        p.m = p.n = p.k = d;
        p.alpha = 1.f; p.beta = 0.f;
        p.A = buf + per * i; p.lda = d;
        p.B = buf + per * i + d * d; p.ldb = d;
        p.C = buf + per * i + 2 * d * d; p.ldc = d;
    }
    return ps;
}

// Best of two timed runs (after a warm-up) of a plan built with `choice`.
int time_choice(gb_handle_t h, int dev, const std::vector<gb_gemm_problem_t> &ps,
                const int choice[kClasses], void *ws, cudaStream_t s, cudaEvent_t e0,
                cudaEvent_t e1, float *ms) {
    gb_grouped_plan_s *pl = nullptr;
    if (build_plan(h, dev, ps, choice, kPrefAuto, &pl) != GB_OK) return GB_ERR_CUDA;
    int rc = GB_OK;
    *ms = 1e30f;
    for (int rep = 0; rep < 3 && rc == GB_OK; ++rep) {
        cudaEventRecord(e0, s);
        if (run_plan(pl, ws, s) != GB_OK) { rc = GB_ERR_CUDA; break; }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = GB_ERR_CUDA; break; }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) *ms = std::min(*ms, t);
    }
    destroy_plan(pl);
    return rc;
}

// Autotuner: for each size class, time a synthetic group of square problems
// of the class's middle size (geometric mean 2^(c+3.5)) under each candidate
// (SIMT 64x64 tiles, SIMT 128x128 tiles, and the tensor cores in each of the
// three grouped configurations: tile width, row width, stage count and CTAs
// per SM, see tc_body.cuh) and keep the fastest.
// A class timed alone does not see that its SIMT part and the tensor-core
// part of a mixed group share the SMs (a SIMT CTA does not fit beside two
// tensor-core CTAs), so the per-class choice is then checked on one mixed
// synthetic group (equal problem counts per class, as in a log-uniform
// group) against routing every class to the tensor cores, in the classes'
// configurations or all in configuration 0 (a class timed alone favours
// the one-CTA-per-SM configurations, which give up parallelism in a mixed
// group): the fastest of the three routings is kept. Runs once per handle, on a private stream, with scratch memory
// freed afterwards; the result is stored in the handle.
int autotune(gb_handle_t h, int dev) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GB_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = GB_OK;
    void *ws = nullptr;
    if (cudaMalloc(&ws, 256) != cudaSuccess) rc = GB_ERR_CUDA;
    for (int c = 0; c < kClasses && rc == GB_OK; ++c) {
        const int64_t d = (int64_t)llround(pow(2.0, c + 3.5));
        // enough problems for about two waves of 128 x 128 tiles, bounded in memory
        const int64_t tiles = ((d + 127) / 128) * ((d + 127) / 128);
        int64_t g = std::max<int64_t>(16, (2 * (int64_t)h->sm_count + tiles - 1) / tiles);
        g = std::min<int64_t>(g, std::max<int64_t>(4, (int64_t)(256ll << 20) / (12 * d * d)));
        float *buf = nullptr;
        const size_t per = (size_t)(3 * d * d);
        if (cudaMalloc(&buf, per * g * sizeof(float)) != cudaSuccess) { rc = GB_ERR_CUDA; break; }
        cudaMemsetAsync(buf, 0x3e, per * g * sizeof(float), s);   // values near 0.19
        const std::vector<gb_gemm_problem_t> ps = synthetic(buf, g, d, 0);
        float best = 1e30f;
        int best_ch = 1;
        for (int ch = 0; ch < kChoices && rc == GB_OK; ++ch) {
            int choice[kClasses];
            for (int q = 0; q < kClasses; ++q) choice[q] = ch;
            float ms = 1e30f;
            rc = time_choice(h, dev, ps, choice, ws, s, e0, e1, &ms);
            if (ms < best) { best = ms; best_ch = ch; }
        }
        cudaFree(buf);
        h->grouped_choice[c] = best_ch;
    }
    // The mixed check: 512 uneven problems with M, N and K each drawn
    // log-uniformly from [8, 1024] (a fixed xorshift sequence), as grouped
    // workloads of uneven sizes come, in about 0.5 GB of scratch. Needed
    // unless every class already chose the tensor cores in configuration 0.
    bool any_other = false;
    for (int c = 0; c < kClasses; ++c) any_other |= h->grouped_choice[c] != 2;
    // a mixed plan runs its two parts concurrently only on the side stream
    if (rc == GB_OK && any_other && !ensure_side(h)) rc = GB_ERR_CUDA;
    if (rc == GB_OK && any_other) {
        std::vector<gb_gemm_problem_t> mix(512);
        std::vector<float *> bufs;
        uint64_t x = 0x9e3779b97f4a7c15ull;
        auto dim = [&]() {
            x ^= x << 13; x ^= x >> 7; x ^= x << 17;
            const double u = (double)(x >> 11) / 9007199254740992.0;   // [0, 1)
            return (int64_t)llround(pow(2.0, 3.0 + 7.0 * u));
        };
        size_t total = 0;
        for (gb_gemm_problem_t &p : mix) {
            p.m = dim(); p.n = dim(); p.k = dim();
            total += (size_t)(p.m * p.k + p.k * p.n + p.m * p.n);
        }
        float *buf = nullptr;
        if (cudaMalloc(&buf, total * sizeof(float)) != cudaSuccess) rc = GB_ERR_CUDA;
        else {
            bufs.push_back(buf);
            cudaMemsetAsync(buf, 0x3e, total * sizeof(float), s);
            size_t off = 0;
            for (size_t i = 0; i < mix.size(); ++i) {
                gb_gemm_problem_t &p = mix[i];
                p.transa = (i & 1) ? 'T' : 'N';
                p.transb = (i & 2) ? 'T' : 'N';
                p.alpha = 1.f; p.beta = 0.f;
                p.A = buf + off; p.lda = p.transa == 'T' ? p.k : p.m; off += (size_t)(p.m * p.k);
                p.B = buf + off; p.ldb = p.transb == 'T' ? p.n : p.k; off += (size_t)(p.k * p.n);
                p.C = buf + off; p.ldc = p.m; off += (size_t)(p.m * p.n);
            }
        }
        if (rc == GB_OK) {
            // three routings of the mixed group: as tuned per class; every
            // class on the tensor cores in its tuned configuration (SIMT
            // classes in configuration 0); every class in configuration 0
            int cand[3][kClasses];
            for (int c = 0; c < kClasses; ++c) {
                cand[0][c] = h->grouped_choice[c];
                cand[1][c] = cand[0][c] >= 2 ? cand[0][c] : 2;
                cand[2][c] = 2;
            }
            float best_t = 1e30f;
            int best = 0;
            for (int i = 0; i < 3 && rc == GB_OK; ++i) {
                float t = 1e30f;
                rc = time_choice(h, dev, mix, cand[i], ws, s, e0, e1, &t);
                if (t < best_t) { best_t = t; best = i; }
            }
            if (rc == GB_OK)
                for (int c = 0; c < kClasses; ++c) h->grouped_choice[c] = cand[best][c];
        }
        for (float *b : bufs) cudaFree(b);
    }
    cudaFree(ws);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc == GB_OK) {
        h->grouped_tuned = true;
        gb::tuning_autosave(h);
    }
    return rc;
}

}  // namespace

int gb::grouped_autotune(gb_handle_t h) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != h->device) return GB_ERR_HANDLE;
    return autotune(h, dev);
}

extern "C" GB_API int gb_tune_grouped(gb_handle_t h) {
    if (!h || h->magic != gb::kHandleMagic) return GB_ERR_HANDLE;
    return gb::grouped_autotune(h);
}

extern "C" {

GB_API int gb_sgemm_grouped_plan(gb_handle_t h, gb_algo_t algo, int64_t count,
                                 const gb_gemm_problem_t *hp, gb_grouped_plan_t *plan,
                                 size_t *ws_bytes, int64_t *bad_index) {
    using namespace gb;
    if (plan) *plan = nullptr;
    if (bad_index) *bad_index = -1;
    if (!plan || !ws_bytes || count < 0 || (count > 0 && !hp)) return GB_ERR_ARG;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != h->device) return GB_ERR_HANDLE;
    if (count > (int64_t)1 << 30) return GB_ERR_UNSUPPORTED;
    std::vector<gb_gemm_problem_t> ps;
    ps.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const gb_gemm_problem_t &p = hp[i];
        int rc = check_problem(p);
        if (rc) {
            if (bad_index) *bad_index = i;
            return rc;
        }
        const bool scale_only = p.alpha == 0.f || p.k == 0;
        const bool quick = p.m == 0 || p.n == 0 || (scale_only && p.beta == 1.f);
        if (!quick && (!p.C || (!scale_only && (!p.A || !p.B)))) {
            if (bad_index) *bad_index = i;
            return GB_ERR_ARG;
        }
        ps.push_back(p);
    }
    int choice[kClasses];
    if (algo == GB_ALGO_AUTO) {
        if (!h->grouped_tuned) {
            int rc = autotune(h, dev);
            if (rc) return rc;
        }
        for (int c = 0; c < kClasses; ++c) choice[c] = h->grouped_choice[c];
    } else {
        // SIMT: 64x64 tiles for the three smallest classes, else 128x128;
        // a split algorithm: every problem with K >= 9 on the tensor cores,
        // in the configuration the tuner chose for its class if the handle
        // has tuned (or loaded) one, else configuration 0
        for (int c = 0; c < kClasses; ++c)
            choice[c] = algo == GB_ALGO_SIMT ? (c < 3 ? 0 : 1)
                        : (h->grouped_tuned && h->grouped_choice[c] >= 2 ? h->grouped_choice[c] : 2);
    }
    // the scaled FP16 split has no grouped kernel: its problems take TF32X3,
    // whose per-product error is of the same order (3 * 2^-22)
    const int pref = (algo == GB_ALGO_SPLIT_TF32X3 || algo == GB_ALGO_SPLIT_FP16X3) ? 0
                   : algo == GB_ALGO_SPLIT_BF16X3 ? 1
                   : algo == GB_ALGO_SPLIT_BF16X6 ? 2 : algo == GB_ALGO_SPLIT_BF16X9 ? 3
                   : kPrefAuto;
    gb_grouped_plan_s *pl = nullptr;
    int rc = build_plan(h, dev, ps, choice, pref, &pl);
    if (rc) return rc;
    if (pl->tc_nitems > 0 && pl->nitems > 0 && !ensure_side(h)) {
        destroy_plan(pl);
        return GB_ERR_CUDA;
    }
    *ws_bytes = 256;         // the SIMT work counter
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
    if (plan->nitems == 0 && plan->tc_nitems == 0) return GB_OK;
    if (!workspace || ws_bytes < 256 || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return GB_ERR_WORKSPACE;
    return run_plan(plan, workspace, static_cast<cudaStream_t>(stream));
}

GB_API int gb_sgemm_grouped_destroy(gb_grouped_plan_t plan) {
    if (!plan) return GB_OK;
    if (plan->magic != kPlanMagic) return GB_ERR_PLAN;
    destroy_plan(plan);
    return GB_OK;
}

}  // extern "C"
