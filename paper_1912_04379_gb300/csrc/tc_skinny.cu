// Split-precision SGEMM for skinny products: one operand has at most 64 rows
// (M <= 64 or N <= 64) and the other is long. Such a product is bound by
// reading the long operand once from HBM; the two-pass path would read it as
// FP32, write its terms and read the terms again, three times the bytes.
//
// The long operand X (op(B)^T when M is short, op(A) when N is short) comes
// by TMA as FP32 tiles of 128 rows x 32 k straight from the caller's storage,
// and eight converter warps split each tile in shared memory into its BF16
// terms, laid out as tcgen05.mma reads them (the paper's re-buffering of B',
// Sec. 3, done between L2 and the tensor cores). The short operand Y is split
// once by the pack pass (a few MB); the producer brings its terms by TMA into
// the same stage as the FP32 tile. The MMA forms the 128 x 64 tile D[x, y] =
// sum_k X[x, k] Y[y, k]: X rows on the TMEM lanes, Y rows on 64 columns.
// The products of one X term with all the Y terms it pairs with go into one
// MMA, the Y terms stacked along N (they lie one after another in shared
// memory): for three terms X0 [Y0; Y1; Y2] (N = 192), X1 [Y0; Y1] (N = 128)
// and X2 Y0 (N = 64), three MMAs per 16 k instead of six. Column group j of
// the accumulator then holds the products with Y_j, and the epilogue adds
// the groups in order. A narrow MMA costs about as much to issue as a wide
// one, so the count of MMA instructions, not their width, set the pace.
// The converters work in two groups of four warps that take alternate
// k-blocks, so that one group's wait, load and signalling latency overlaps
// the other's conversion.
//
// Work: the (tile, k-block) iteration space is cut into one contiguous range
// of equal length per CTA (stream-K), so every SM streams the same number of
// X bytes whatever the shape. A tile whose k-blocks fall to several CTAs is
// finished by the last of them: each writes its raw partial sum to a slot
// fixed by the partition, counts itself in at the tile's counter, and the
// one that completes the count adds the slots in slot order and writes C.
// The order of the additions is therefore fixed: the result does not depend
// on timing.
//
// Warps: 0 TMA producer (X), 1 TMEM owner + MMA issuer, 2..5 epilogue,
// 6..13 converters (448 threads, one CTA per SM). Every wait is bounded as in
// the other tensor-core kernels.
#include "f32_tile.cuh"

namespace gb {
namespace {

using namespace tcx;
using namespace fx;

constexpr int SK_YN = 64;                      // MMA N: rows of the short operand
constexpr int SK_NCONV = 8;                    // converter warps
constexpr int SK_GROUPS = 2;                   // converter groups, alternate k-blocks
constexpr int SK_GW = SK_NCONV / SK_GROUPS;    // warps per group
constexpr int SK_CONV0 = 6;                    // first converter warp
constexpr int SK_THREADS = (SK_CONV0 + SK_NCONV) * 32;
constexpr int SK_SLOT = BM * SK_YN;            // floats in one partial-sum slot

template <int MODE>     // 1: BF16 x 2 terms, 3 products; 2: x 3 terms, 6 products; 3: x 3 terms, 9
struct SkCfg {
    static constexpr int PARTS = MODE >= 2 ? 3 : 2;
    // k per stage: KH sub-blocks of 32 (the TMA boxes and the 64-byte rows
    // of the Y terms are 32 k wide); two for the two-term split, whose
    // narrower accumulators leave tensor memory for 64-k stages: per k, the
    // MMA issuer's waits and commits then cost half
    static constexpr int KH = MODE >= 2 ? 1 : 2;
    static constexpr int SKB = KH * FBK;
    static constexpr int F32_BYTES = BM * FBK * 4;          // one FP32 X sub-tile
    static constexpr int X_BYTES = KH * F32_BYTES;
    static constexpr int Y_OP = SK_YN * 64;                 // one Y term: 64 rows of 64 B
    // A shared-memory stage: the FP32 X sub-tiles (h at +h*F32_BYTES), then
    // the Y terms (sub-block h, term p at +X_BYTES + (h*PARTS + p)*Y_OP).
    static constexpr int STAGE = X_BYTES + KH * PARTS * Y_OP;
    static constexpr int STAGES = MODE >= 2 ? 8 : 4;
    // TMEM: two accumulators of PARTS column groups (products with Y_0,
    // Y_1, ...), then the X-term stages: sub-block h, term p at 16 (h*PARTS
    // + p) columns (32 BF16 of K, two per column)
    static constexpr int ACC_COLS = PARTS * SK_YN;
    static constexpr int XCOLS = KH * PARTS * (FBK / 2);
    static constexpr int T_STAGES = MODE >= 2 ? 2 : 4;
    static constexpr int TMEM_COLS = 512;
    // equal ring lengths: one MMA commit per k-block releases both stages
    static constexpr bool SHARED_RELEASE = T_STAGES == STAGES;
    static constexpr int NBARS = 2 * STAGES + 2 * T_STAGES + 5;
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE + 8 * NBARS + 16;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
    static_assert(2 * ACC_COLS + T_STAGES * XCOLS <= TMEM_COLS, "tensor memory");
    // Every stage belongs to one group (stage counts a multiple of the group
    // count): a group then waits on a stage's barrier only one phase ahead
    // of the last phase it saw there, so a parity wait cannot pass on an
    // older phase of the same parity.
    static_assert(STAGES % SK_GROUPS == 0 && T_STAGES % SK_GROUPS == 0, "stage ownership");
    static_assert(STAGE % 1024 == 0 && F32_BYTES % 1024 == 0, "swizzle atoms stay aligned");
};

// The stream-K partition: L = tiles * nkb iterations, CTA c takes
// [lo(c), lo(c + 1)); owner(g) is the CTA whose range holds iteration g.
struct SkPart {
    int64_t L;
    int64_t nkb;
    int G;
    __device__ __forceinline__ int64_t lo(int c) const { return (int64_t)c * L / G; }
    __device__ __forceinline__ int owner(int64_t g) const { return (int)(((g + 1) * G - 1) / L); }
};

struct SkArgs {
    int64_t R;                    // rows of X
    int64_t Yrows;                // rows of Y (<= 64)
    float alpha, beta;
    float *C;
    int64_t ldc;
    int x_is_b;                   // 1: X = op(B)^T, D[x, y] = C[y, x]; 0: X = op(A), D[x, y] = C[x, y]
    int xkc;                      // X is K-contiguous in storage
    int cvec;                     // x_is_b and rows of C 16-byte aligned (C and ldc): float4 stores
    float *slots;                 // partial sums, (tiles + G) slots of 128 x 64
    unsigned *count;              // per tile, zero at launch
};

// Named barrier 1 over the four epilogue warps (barrier 0 is __syncthreads).
__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// AND of `pred` over the epilogue threads; also synchronises them.
__device__ __forceinline__ bool epi_all(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
    return r != 0;
}

// C for NV values of row x of the tile, columns y0 .. y0 + NV - 1: C[y, x]
// (x_is_b) or C[x, y], y < Yrows; C <- alpha * v + beta * C (C not read
// when beta == 0), the split-K reduction's arithmetic. With x_is_b the
// values are contiguous in C, 16-byte vectors when cvec (y0 % 4 == 0).
template <int NV>
__device__ __forceinline__ void sk_store_c(const SkArgs &a, int64_t x, int y0, const float (&v)[NV]) {
    if (x >= a.R) return;
    const int64_t step = a.x_is_b ? 1 : a.ldc;
    float *p = (a.x_is_b ? a.C + x * a.ldc : a.C + x) + y0 * step;
    const int ny = (int)a.Yrows - y0;
    if (a.cvec) {
#pragma unroll
        for (int y = 0; y < NV; y += 4) {
            if (y + 3 < ny) {
                float4 *q = reinterpret_cast<float4 *>(p + y);
                float4 r = make_float4(a.alpha * v[y], a.alpha * v[y + 1], a.alpha * v[y + 2],
                                       a.alpha * v[y + 3]);
                if (a.beta != 0.f) {
                    const float4 c = *q;
                    r = make_float4(fmaf(a.alpha, v[y], a.beta * c.x), fmaf(a.alpha, v[y + 1], a.beta * c.y),
                                    fmaf(a.alpha, v[y + 2], a.beta * c.z), fmaf(a.alpha, v[y + 3], a.beta * c.w));
                }
                *q = r;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (y + e < ny) p[y + e] = a.beta == 0.f ? a.alpha * v[y + e] : fmaf(a.alpha, v[y + e], a.beta * p[y + e]);
            }
        }
        return;
    }
    if (a.beta == 0.f) {
#pragma unroll
        for (int y = 0; y < NV; ++y)
            if (y < ny) p[y * step] = a.alpha * v[y];
    } else {
#pragma unroll
        for (int y = 0; y < NV; ++y)
            if (y < ny) p[y * step] = fmaf(a.alpha, v[y], a.beta * p[y * step]);
    }
}

template <int MODE>
__global__ void __launch_bounds__(SK_THREADS, 1)
tc_skinny_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                 const SkArgs a, const SkPart P, DeviceState *dstate, uint64_t limit_ns) {
    using CF = SkCfg<MODE>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    // stage s at base + s*STAGE: the FP32 X tile at +0, the Y terms at
    // +F32_BYTES + p*Y_OP; then the barriers
    const uint32_t bar_base = base + CF::STAGES * CF::STAGE;
    uint8_t *gbar = gbase + CF::STAGES * CF::STAGE;
    constexpr int F = CF::STAGES, T = CF::T_STAGES;
    // in_full: TMA landed X and Y; in_empty: the group's converters used X
    // and the MMAs read Y; t_full: X terms in TMEM; t_empty: MMAs read them
    auto in_full = [&](int s) { return bar_base + 8u * s; };
    auto in_empty = [&](int s) { return bar_base + 8u * (F + s); };
    auto t_full = [&](int s) { return bar_base + 8u * (2 * F + s); };
    auto t_empty = [&](int s) { return bar_base + 8u * (2 * F + T + s); };
    auto acc_full = [&](int b) { return bar_base + 8u * (2 * F + 2 * T + b); };
    auto acc_empty = [&](int b) { return bar_base + 8u * (2 * F + 2 * T + 2 + b); };
    const uint32_t drain_bar = bar_base + 8u * (2 * F + 2 * T + 4);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(gbar + 8 * CF::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbar + 8 * CF::NBARS + 4);
    volatile int *last_flag = reinterpret_cast<volatile int *>(gbar + 8 * CF::NBARS + 8);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    WaitCtx w{abort_flag, dstate, limit_ns};

    if (threadIdx.x == 0) {
        for (int s = 0; s < F; ++s) {
            mbar_init(in_full(s), 1);
            mbar_init(in_empty(s), SK_GW + (CF::SHARED_RELEASE ? 0 : 1));
        }
        for (int s = 0; s < T; ++s) {
            mbar_init(t_full(s), SK_GW);
            mbar_init(t_empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), 4);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        *last_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_tmap(&mapX);
        prefetch_tmap(&mapY);
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), CF::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    const int64_t nkb = P.nkb;
    const int64_t g0 = P.lo(blockIdx.x), g1 = P.lo(blockIdx.x + 1);

    if (warp == 0) {
        if (lane == 0) {
            // ------------- TMA producer: FP32 tiles of X, terms of Y -------------
            // The kernel may start while the pack of Y (the launch before it)
            // still runs: the first F stages' X tiles go out at once, then
            // the producer waits for that grid (griddepcontrol.wait; a no-op
            // when the kernel was not launched as its dependent) and issues
            // their Y terms; from then on X and Y together. Each stage's
            // expect_tx counts X and Y, so in_full completes only with both.
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            int64_t t = g0 / nkb;
            int kb = (int)(g0 - t * nkb);
            const int64_t early = (g1 - g0) < F ? (g1 - g0) : F;   // stages whose Y waits
            auto load_x = [&](uint32_t dst, int st, int64_t tt, int kk) {
#pragma unroll
                for (int h = 0; h < CF::KH; ++h) {
                    const int k0 = kk * CF::SKB + h * FBK;
                    if (a.xkc) tma_load_2d(dst + h * CF::F32_BYTES, &mapX, in_full(st), k0, (int)(tt * BM));
                    else       tma_load_2d(dst + h * CF::F32_BYTES, &mapX, in_full(st), (int)(tt * BM), k0);
                }
            };
            auto load_y = [&](uint32_t dst, int st, int kk) {
#pragma unroll
                for (int h = 0; h < CF::KH; ++h)
#pragma unroll
                    for (int p = 0; p < CF::PARTS; ++p)
                        tma_load_3d(dst + CF::X_BYTES + (h * CF::PARTS + p) * CF::Y_OP, &mapY, in_full(st),
                                    kk * CF::SKB + h * FBK, 0, p);
            };
            // the first stages are empty: X only
            {
                int64_t tt = t;
                int kk = kb;
                for (int64_t i = 0; i < early; ++i, ++kk) {
                    if (kk == nkb) { kk = 0; ++tt; }
                    const uint32_t dst = base + (int)i * CF::STAGE;
                    mbar_arrive_expect_tx(in_full((int)i), CF::STAGE);
                    load_x(dst, (int)i, tt, kk);
                }
                asm volatile("griddepcontrol.wait;" ::: "memory");
                kk = kb;
                for (int64_t i = 0; i < early; ++i, ++kk) {
                    if (kk == nkb) kk = 0;
                    load_y(base + (int)i * CF::STAGE, (int)i, kk);
                    issued |= 1u << i;
                }
            }
            for (int64_t g = g0; g < g1; ++g, ++kb) {
                if (kb == nkb) { kb = 0; ++t; }
                if (g - g0 >= early) {
                    if (!wait_bounded(w, in_empty(s), ph ^ 1u, kSiteProducerEmpty)) break;
                    // with one ring length, the MMAs' release of the k-block's
                    // TMEM stage also releases its input stage (same index)
                    if (CF::SHARED_RELEASE && !wait_bounded(w, t_empty(s), ph ^ 1u, kSiteProducerEmpty)) break;
                    const uint32_t dst = base + s * CF::STAGE;
                    mbar_arrive_expect_tx(in_full(s), CF::STAGE);
                    load_x(dst, s, t, kb);
                    load_y(dst, s, kb);
                    issued |= 1u << s;
                }
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == F) { s = 0; ph ^= 1u; }
            }
            for (int i = 0; i < F; ++i) {
                if (!(issued & (1u << i))) continue;
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(in_full(i), (last_par >> i) & 1u)) {
                    if (global_ns() - t0 > kDrainLimitNs) { record_timeout(w, kSiteDrain); break; }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int s = 0, st = 0, acc = 0;
            uint32_t ph = 0, pht = 0, acc_ph = 0;
            bool ok = true;
            for (int64_t t = g0 / nkb; t * nkb < g1 && ok; ++t) {
                const int kb0 = (int)((g0 > t * nkb ? g0 : t * nkb) - t * nkb);
                const int kb1 = (int)((g1 < (t + 1) * nkb ? g1 : (t + 1) * nkb) - t * nkb);
                if (!wait_bounded(w, acc_empty(acc), acc_ph ^ 1u, kSiteMmaAccEmpty)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * CF::ACC_COLS);
                uint32_t accumulate = 0;
                for (int kb = kb0; kb < kb1; ++kb) {
                    // The converters of this k-block waited for its stage to
                    // land (X and Y alike) before they signalled t_full, so
                    // that one wait orders the Y bytes before the MMAs too.
                    if (!wait_bounded(w, t_full(st), pht, kSiteMmaFull)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xt = tmem_base + (uint32_t)(2 * CF::ACC_COLS + st * CF::XCOLS);
                    // X term i (from TMEM) with Y terms 0 .. NY(i)-1 stacked along
                    // N: the pairs of the split (i + j <= PARTS - 1; all nine
                    // pairs for BF16 x 3 terms with 9 products)
#pragma unroll
                    for (int h = 0; h < CF::KH; ++h)
#pragma unroll
                    for (int i = 0; i < CF::PARTS; ++i) {
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            // K = 16 per MMA: 8 TMEM columns of X, 32 bytes of a Y row
                            const uint32_t xa = xt + (uint32_t)((h * CF::PARTS + i) * (FBK / 2) + ks * 8);
                            const uint64_t yd = smem_desc<64>(base + s * CF::STAGE + CF::X_BYTES +
                                                              h * CF::PARTS * CF::Y_OP + ks * 32);
                            const int ny = MODE == 3 ? CF::PARTS : CF::PARTS - i;
                            if (ny == 3)
                                mma_issue_ta(d_tmem, xa, yd, instr_desc<kFmtBF16, 3 * SK_YN>(), accumulate);
                            else if (ny == 2)
                                mma_issue_ta(d_tmem, xa, yd, instr_desc<kFmtBF16, 2 * SK_YN>(), accumulate);
                            else
                                mma_issue_ta(d_tmem, xa, yd, instr_desc<kFmtBF16, SK_YN>(), accumulate);
                            accumulate = 1;
                        }
                    }
                    mma_commit(t_empty(st));            // X terms read
                    if (!CF::SHARED_RELEASE)
                        mma_commit(in_empty(s));        // Y terms read: the MMA's share of the stage
                    if (++st == T) { st = 0; pht ^= 1u; }
                    if (++s == F) { s = 0; ph ^= 1u; }
                }
                if (!ok) break;
                mma_commit(acc_full(acc));
                if (++acc == 2) { acc = 0; acc_ph ^= 1u; }
            }
            mma_commit(drain_bar);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(drain_bar, 0)) {
                if (global_ns() - t0 > kDrainLimitNs) { record_timeout(w, kSiteDrain); break; }
            }
        }
        __syncwarp();
    } else if (warp < SK_CONV0) {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;                       // TMEM lanes 32q .. 32q + 31
        const int xr = q * 32 + lane;                 // row of the tile
        int acc = 0;
        uint32_t acc_ph = 0;
        for (int64_t t = g0 / nkb; t * nkb < g1; ++t) {
            const int64_t s0 = g0 > t * nkb ? g0 : t * nkb;
            const int64_t s1 = g1 < (t + 1) * nkb ? g1 : (t + 1) * nkb;
            // all four warps go on or all leave: they meet at named barriers below
            if (!epi_all(wait_bounded(w, acc_full(acc), acc_ph, kSiteEpiAccFull))) break;
            tc_fence_after();
            // 16 columns at a time: the column groups' values (products with
            // Y_0, Y_1, ...), added in group order, go to C (the whole K range
            // is here) or to this CTA's partial-sum slot of the tile, laid
            // out [y / 4][row][y % 4]
            const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * CF::ACC_COLS);
            const int64_t x = t * BM + xr;
            const bool whole = s0 == t * nkb && s1 == (t + 1) * nkb;
            float4 *slot = reinterpret_cast<float4 *>(a.slots + (t + blockIdx.x) * SK_SLOT);
#pragma unroll 1
            for (int c = 0; c < SK_YN; c += 16) {
                uint32_t r[3][16];
#pragma unroll
                for (int u = 0; u < CF::PARTS; ++u) tmem_ld16(ta + (uint32_t)(u * SK_YN + c), r[u]);
                if (CF::PARTS == 3) tmem_wait48(r[0], r[1], r[2]);
                else tmem_wait32(r[0], r[1]);
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float z = __uint_as_float(r[0][j]);
#pragma unroll
                    for (int u = 1; u < CF::PARTS; ++u) z = __fadd_rn(z, __uint_as_float(r[u][j]));
                    v[j] = z;
                }
                if (whole) {
                    sk_store_c<16>(a, x, c, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        __stcg(slot + (c / 4 + j) * BM + xr,
                               make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(acc));
            if (++acc == 2) { acc = 0; acc_ph ^= 1u; }
            if (whole) continue;
            // Count in at the tile (release: the barrier orders every epilogue
            // thread's slot stores before the leader's fence and atomic), and
            // learn whether this CTA completes the count (acquire: the fence
            // after the atomic orders the other CTAs' slot stores, which they
            // released the same way, before the loads below).
            epi_sync();
            const int cf = P.owner(t * nkb), cl = P.owner((t + 1) * nkb - 1);
            if (warp == 2 && lane == 0) {
                __threadfence();
                const unsigned old = atomicAdd(a.count + t, 1u);
                __threadfence();
                *last_flag = old == (unsigned)(cl - cf) ? 1 : 0;
            }
            epi_sync();
            if (!*last_flag) continue;
            // the last of the tile's CTAs: add the slots in slot order, 16
            // columns at a time, the loads of up to four slots issued
            // together (each load is an L2 round trip, and this runs in the
            // kernel's tail)
#pragma unroll 1
            for (int yq = 0; yq < SK_YN / 16; ++yq) {
                float u16[16];
#pragma unroll 1
                for (int c0 = cf; c0 <= cl; c0 += 4) {
                    float4 u[4][4];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        if (c0 + cc > cl) break;
                        const float4 *sp = reinterpret_cast<const float4 *>(
                                               a.slots + (t + c0 + cc) * SK_SLOT) + (yq * 4) * BM + xr;
#pragma unroll
                        for (int j = 0; j < 4; ++j) u[cc][j] = __ldcg(sp + j * BM);
                    }
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        if (c0 + cc > cl) break;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float uu[4] = {u[cc][j].x, u[cc][j].y, u[cc][j].z, u[cc][j].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                u16[4 * j + e] = (c0 + cc == cf) ? uu[e] : __fadd_rn(u16[4 * j + e], uu[e]);
                        }
                    }
                }
                sk_store_c<16>(a, x, 16 * yq, u16);
            }
        }
    } else {
        // ---------------- converters (warps 6..13, two groups) ----------------
        // Group gi takes the k-blocks at even (gi = 0) or odd (gi = 1)
        // positions of this CTA's range. Each thread converts one row of the
        // tile, the TMEM lane its warp may access (32 (warp % 4) + lane): it
        // waits for a free TMEM stage, then per 32-k sub-block reads its FP32
        // values, splits them and stores the terms there; it waits for the
        // stores and signals; the input stage goes back only now, after its
        // values were used.
        const int ct = threadIdx.x - SK_CONV0 * 32;
        const int gi = ct / (32 * SK_GW);
        const int row = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        for (int64_t it = gi; it < g1 - g0; it += SK_GROUPS) {
            const int s = (int)(it % F), st = (int)(it % T);
            const uint32_t ph = (uint32_t)(it / F) & 1u, pht = (uint32_t)(it / T) & 1u;
            if (!__all_sync(0xffffffffu, wait_bounded(w, in_full(s), ph, kSiteConvert))) break;
            if (!__all_sync(0xffffffffu, wait_bounded(w, t_empty(st), pht ^ 1u, kSiteConvert))) break;
            tc_fence_after();
            const uint32_t xt = tmem_base + lane_base + (uint32_t)(2 * CF::ACC_COLS + st * CF::XCOLS);
#pragma unroll
            for (int h = 0; h < CF::KH; ++h) {
                const float *fxp = reinterpret_cast<const float *>(gbase + s * CF::STAGE + h * CF::F32_BYTES);
                float v[FBK];
#pragma unroll
                for (int c = 0; c < FBK / 8; ++c) read8<BM>(fxp, a.xkc != 0, row, c, v + 8 * c);
                // terms, two K values per 32-bit column (the lower K in the low
                // half); one branch for all 32 values: the exact scalar split
                // only when one of them is non-finite or near overflow
                uint32_t tw[CF::PARTS][FBK / 2];
                if (max_abs_bits(v) < kBf16FastLimit) {
#pragma unroll
                    for (int e = 0; e < FBK / 2; ++e) {
                        uint32_t pr[CF::PARTS];
                        split2_bf16_fast<CF::PARTS>(v[2 * e], v[2 * e + 1], pr);
#pragma unroll
                        for (int p = 0; p < CF::PARTS; ++p) tw[p][e] = pr[p];
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < FBK / 2; ++e) {
                        uint32_t pr[CF::PARTS];
                        split2_bf16<CF::PARTS>(v[2 * e], v[2 * e + 1], pr);
#pragma unroll
                        for (int p = 0; p < CF::PARTS; ++p) tw[p][e] = pr[p];
                    }
                }
#pragma unroll
                for (int p = 0; p < CF::PARTS; ++p)
                    tmem_st16(xt + (uint32_t)((h * CF::PARTS + p) * (FBK / 2)), tw[p]);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(t_full(st));
                mbar_arrive(in_empty(s));
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, CF::TMEM_COLS);
}

// 3-D map over the packed short operand, [term][row][kpad] BF16 with terms
// part_stride elements apart: a box is 32 k x 64 rows of one term, 64-byte
// rows with the 64-byte swizzle. Rows past Yrows and k past K read as 0.
bool make_terms_map(CUtensorMap *map, const void *ptr, int64_t k, int64_t rows, int64_t kpad,
                    int parts, int64_t part_stride) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)parts};
    cuuint64_t strides[2] = {(cuuint64_t)(kpad * 2), (cuuint64_t)(part_stride * 2)};
    cuuint32_t box[3] = {(cuuint32_t)FBK, (cuuint32_t)SK_YN, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int MODE>
cudaError_t launch_skinny_mode(const SkinnyArgs &h, cudaStream_t s) {
    using CF = SkCfg<MODE>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        e = cudaFuncSetAttribute(tc_skinny_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    // X: op(B)^T (stored K x N unless B is transposed) or op(A) (stored
    // M x K unless A is transposed); K-contiguous storage is read along K.
    const bool xkc = h.x_is_b ? !h.tb : h.ta;
    const float *X = h.x_is_b ? h.B : h.A;
    const int64_t ldx = h.x_is_b ? h.ldb : h.lda;
    const int64_t R = h.x_is_b ? h.n : h.m, Yrows = h.x_is_b ? h.m : h.n;
    alignas(64) CUtensorMap mx, my;
    if (!make_f32_map(&mx, X, xkc ? h.k : R, xkc ? R : h.k, ldx, xkc, BM) ||
        !make_terms_map(&my, h.Yp, h.k, Yrows, h.kpad, CF::PARTS, Yrows * h.kpad))
        return cudaErrorNotSupported;
    const int64_t tiles = (R + BM - 1) / BM;
    const int64_t nkb = (h.k + CF::SKB - 1) / CF::SKB;
    int G = h.sm_count > 0 ? h.sm_count : 1;
    if (G > kSkinnyMaxCtas) G = kSkinnyMaxCtas;
    if (tiles * nkb < G) G = (int)(tiles * nkb);
    // the slots and counters, as skinny_ws_bytes lays them out (the
    // counters were zeroed by skinny_clear before the pack of Y)
    float *slots = reinterpret_cast<float *>(h.ws);
    unsigned *count = reinterpret_cast<unsigned *>(
        static_cast<char *>(h.ws) + (size_t)(tiles + kSkinnyMaxCtas) * SK_SLOT * sizeof(float));
    const bool cvec = h.x_is_b && !(reinterpret_cast<uintptr_t>(h.C) & 15) && h.ldc % 4 == 0;
    SkArgs a{R, Yrows, h.alpha, h.beta, h.C, h.ldc, h.x_is_b ? 1 : 0, xkc ? 1 : 0, cvec ? 1 : 0,
             slots, count};
    SkPart P{tiles * nkb, nkb, G};
    // launched as the programmatic dependent of the pack of Y before it: the
    // kernel's set-up and first X loads overlap the pack's tail (the
    // producer waits for the pack before it reads Y)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(SK_THREADS);
    cfg.dynamicSmemBytes = CF::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, tc_skinny_kernel<MODE>, mx, my, a, P, h.dstate,
                           (uint64_t)h.wait_limit * 1000ull);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

size_t skinny_ws_bytes(int64_t R) {
    const int64_t tiles = (R + BM - 1) / BM;
    return (size_t)(tiles + kSkinnyMaxCtas) * SK_SLOT * sizeof(float) + (size_t)tiles * sizeof(unsigned);
}

bool skinny_shape(int mode, int64_t m, int64_t n, int64_t k) {
    if (mode < 1 || mode > 3) return false;
    if ((m > SK_YN && n > SK_YN) || k < 256) return false;
    const int64_t R = m > n ? m : n;
    if (R * k < ((int64_t)1 << 22)) return false;
    return R < 2147483647LL && k < 2147483647LL;
}

bool skinny_x_is_b(int64_t m, int64_t n) { return m <= SK_YN && n >= m; }

cudaError_t skinny_clear(const SkinnyArgs &a, cudaStream_t s) {
    const int64_t R = a.x_is_b ? a.n : a.m;
    const int64_t tiles = (R + BM - 1) / BM;
    unsigned *count = reinterpret_cast<unsigned *>(
        static_cast<char *>(a.ws) + (size_t)(tiles + kSkinnyMaxCtas) * SK_SLOT * sizeof(float));
    return cudaMemsetAsync(count, 0, (size_t)tiles * sizeof(unsigned), s);
}

bool skinny_supported(int mode, int64_t m, int64_t n, int64_t k, const float *A, int64_t lda,
                      const float *B, int64_t ldb) {
    if (!skinny_shape(mode, m, n, k)) return false;
    return skinny_x_is_b(m, n) ? f32_tma_ok(B, ldb) : f32_tma_ok(A, lda);
}

cudaError_t launch_tc_skinny(const SkinnyArgs &a, cudaStream_t s) {
    switch (a.mode) {
        case 1: return launch_skinny_mode<1>(a, s);
        case 2: return launch_skinny_mode<2>(a, s);
        case 3: return launch_skinny_mode<3>(a, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace gb
