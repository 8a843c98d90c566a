// The warp-specialised tcgen05 kernel body shared by every tensor-core
// kernel of the library (one GEMM, grouped GEMMs, triangular updates):
// stage configuration, the per-role loops, and the grouped work source.
// A work source supplies num_units() and unit(u, UnitInfo&) (tile, K range,
// tensor maps, output); kTri selects the triangle-masked epilogue.
#pragma once

#include "split_common.cuh"
#include "tc_ptx.cuh"

namespace gb {
namespace tcx {

constexpr int NUM_THREADS = 192;

// ----------------------------------------------------------- the kernel --
// BNX != 0 fixes the tile width; BUDGET_KB is the shared memory the stages
// may take (the one-GEMM kernels: 216 KiB, one CTA per SM). PROMO selects
// promoted accumulation: the MMA warp starts a fresh TMEM accumulator every
// few k-blocks (a chunk of K) and eight epilogue warps add the finished
// chunks, in FP32 with round-to-nearest, into a running sum they keep in
// registers (each warp one TMEM lane quarter and half of the tile's columns).
template <int MODE, int RB, int BNX = 0, int BUDGET_KB = 216, bool PROMO_ = false>
struct Cfg {
    static constexpr int ROW_BYTES = RB;                 // one swizzle row of K
    static constexpr bool TF32 = MODE == 0;
    static constexpr int FMT = MODE == 0 ? kFmtTF32 : MODE == 4 ? kFmtF16 : kFmtBF16;
    // terms per operand: TF32 and BF16 x 2: 2; BF16 x 3: 3; scaled FP16: 3 for
    // op(A) (2^11 h, h, l) and 2 for op(B) (h, l)
    static constexpr int A_PARTS = MODE >= 2 ? 3 : 2;
    static constexpr int B_PARTS = (MODE == 2 || MODE == 3) ? 3 : 2;
    static constexpr int NPAIRS = MODE == 3 ? 9 : MODE == 2 ? 6 : 3;
    // 256 output columns per tile, except 3-term operands with 128-byte rows
    // (a 256-column stage would be 144 KiB: one stage only), which use 128.
    // Wider tiles halve the MMA's re-reads of A from shared memory per flop.
    static constexpr int BN = BNX ? BNX : (MODE >= 2 && RB == 128) ? 128 : 256;
    static constexpr int ELEM = TF32 ? 4 : 2;
    static constexpr int BK = ROW_BYTES / ELEM;          // elements per k-block
    static constexpr int KSTEP_BYTES = 32;               // K per MMA: 16 BF16 / 8 TF32
    static constexpr int KSTEPS = ROW_BYTES / KSTEP_BYTES;
    static constexpr int A_TILE = BM * ROW_BYTES;        // bytes of one term's A tile
    static constexpr int B_TILE = BN * ROW_BYTES;
    static constexpr int STAGE_BYTES = A_PARTS * A_TILE + B_PARTS * B_TILE;
    static constexpr int STAGES = (BUDGET_KB * 1024) / STAGE_BYTES;
    static constexpr int TMEM_COLS = 2 * BN;             // two accumulators
    static constexpr int SMEM_BYTES = 1024 /*align slack*/ + STAGES * STAGE_BYTES + 256;
    static constexpr bool PROMO = PROMO_;
    static constexpr int EPI_WARPS = PROMO ? 8 : 4;
    // Warp roles: 0 = TMA producer, 1 = MMA issuer, then the epilogue warps
    // from EPI_WARP0. The promoted kernel runs three warpgroups (warps 2-3
    // idle) so that it can move registers between them (setmaxnreg, which
    // acts on whole warpgroups): 56 per thread in warpgroup 0, 224 in the
    // two epilogue warpgroups, which hold the running sums.
    static constexpr int EPI_WARP0 = PROMO ? 4 : 2;
    static constexpr int THREADS = 32 * (EPI_WARP0 + EPI_WARPS);
    static constexpr int ECOLS = BN * 4 / EPI_WARPS;     // columns of one epilogue warp
    static constexpr int REG_LOW = 56, REG_HIGH = 224;   // promoted: per-thread registers
    // registers the promoted kernel must be launched with (per thread) so
    // that the split fits: 128 * REG_LOW + 256 * REG_HIGH <= THREADS * this
    static constexpr int REG_LAUNCH_MIN = (128 * REG_LOW + 256 * REG_HIGH + THREADS - 1) / THREADS;
    static_assert(!PROMO || (ECOLS % 64 == 0 && ECOLS <= 128), "promoted epilogue columns");
    static_assert(!PROMO || THREADS == 384, "promoted kernel: three warpgroups");
    static_assert(STAGES >= 2, "need at least two stages");
    static_assert(SMEM_BYTES <= 232448, "opt-in shared memory per block");
    static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM columns");
};

// Many GEMMs: units are the planned (problem, tile) items; each problem has
// its own tensor maps (in device global memory) and output.
template <int BN, int BK>
struct GroupSource {
    static constexpr bool kTri = false;
    static constexpr int kEpi = 0;
    const TcProblem *probs;
    const TcItem *items;
    int64_t nitems;
    __device__ __forceinline__ int64_t num_units() const { return nitems; }
    __device__ __forceinline__ void unit(int64_t u, UnitInfo &ui) const {
        const TcItem it = items[u];
        const TcProblem &P = probs[it.prob];
        ui.ma = P.mapA; ui.mb = P.mapB;
        ui.M = P.m; ui.N = P.n;
        ui.tm = it.tm; ui.tn = it.tn;
        ui.kb0 = 0;
        ui.kb1 = (int)((P.k + BK - 1) / BK);
        ui.alpha = P.alpha; ui.beta = P.beta;
        ui.dst = P.C; ui.ldd = P.ldc;
        ui.raw = false;
    }
};

// Grouped runs, three configurations the autotuner chooses between per size
// class of a problem:
//   V = 0: 128 x 128 tiles of 64-byte rows in 96 KiB of stages, so that two
//          CTAs share an SM (two 256-column TMEM allocations, 2 x 99.6 KB of
//          shared memory): many small tiles are latency-bound, and a second
//          CTA per SM runs its own load / MMA / epilogue pipeline beside the
//          first;
//   V = 1: 128 x 256 tiles of 64-byte rows, 216 KiB of stages, one CTA per SM
//          (the long-K configuration of one GEMM: half the operand re-reads
//          per flop);
//   V = 2: 128 x 128 tiles of 128-byte rows, 216 KiB of stages, one CTA per SM
//          (twice the K per stage: fewer hand-offs per k).
constexpr int kGroupedConfigs = 3;
template <int MODE, int V>
struct GroupedCfgV;
template <int MODE>
struct GroupedCfgV<MODE, 0> : Cfg<MODE, 64, 128, 96> { static constexpr int CTAS = 2; };
template <int MODE>
struct GroupedCfgV<MODE, 1> : Cfg<MODE, 64, 256, 216> { static constexpr int CTAS = 1; };
template <int MODE>
struct GroupedCfgV<MODE, 2> : Cfg<MODE, 128, 128, 216> { static constexpr int CTAS = 1; };
template <int MODE>
using GroupedCfg = GroupedCfgV<MODE, 0>;

// Promoted accumulation for one GEMM: 128 x 256 tiles of 64-byte rows (the
// long-K configuration of the plain kernel), 384 threads. The scaled FP16
// split (56 KiB per stage) takes 224 KiB: four stages.
template <int MODE>
using PromoCfg = Cfg<MODE, 64, 256, MODE == 4 ? 224 : 216, true>;

// Stores one epilogue warp's part of a unit's result from registers: row
// tm*128 + 32q + lane, the EC columns from tn*BN + hcol, value v[j] for
// column j. C <- a*v + beta*C (C not read when beta == 0), or a*v for a
// split-K partial; a is alpha (1 for a partial), times an exact power of two
// for the scaled FP16 split. Same arithmetic as store_tile.
template <int BN, int EC>
__device__ __forceinline__ void store_regs(const UnitInfo &ui, const float (&v)[EC], int hcol,
                                           int q, int lane, float a) {
    const int64_t M = ui.M, N = ui.N, ldd = ui.ldd;
    const bool part = ui.raw;
    const float beta = part ? 0.f : ui.beta;
    const int64_t row = ui.tm * BM + q * 32 + lane;
    const int64_t col0 = ui.tn * BN + hcol;
    float *colp = ui.dst + row + col0 * ldd;
    if ((ui.tm * BM + BM <= M) && (col0 + EC <= N)) {
        if (beta == 0.f) {
#pragma unroll
            for (int j = 0; j < EC; ++j) { *colp = a * v[j]; colp += ldd; }
        } else {
            // the chunk's C values are all read before its first store (a
            // store may alias a later load)
#pragma unroll
            for (int c = 0; c < EC; c += 16) {
                float cv[16];
                const float *qc = colp;
#pragma unroll
                for (int j = 0; j < 16; ++j) { cv[j] = *qc; qc += ldd; }
#pragma unroll
                for (int j = 0; j < 16; ++j) { *colp = fmaf(a, v[c + j], beta * cv[j]); colp += ldd; }
            }
        }
        return;
    }
    if (row >= M || col0 >= N) return;
    const int ncol = (int)(N - col0 < EC ? N - col0 : EC);
#pragma unroll
    for (int j = 0; j < EC; ++j) {
        if (j < ncol) {
            float *p = colp + (int64_t)j * ldd;
            *p = beta != 0.f ? fmaf(a, v[j], beta * *p) : a * v[j];
        }
    }
}

template <int MODE, int RB, class Src, class CF = Cfg<MODE, RB>>
__device__ __forceinline__ void tc_body(const Src &src, DeviceState *dstate, uint64_t limit_ns) {
    static_assert(CF::ROW_BYTES == RB, "configuration row width");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    // [stages][term][A tile] then [stages][term][B tile]
    const uint32_t a_smem = base;
    const uint32_t b_smem = base + CF::STAGES * CF::A_PARTS * CF::A_TILE;
    const uint32_t bar_base = base + CF::STAGES * CF::STAGE_BYTES;
    uint8_t *gbar = gbase + CF::STAGES * CF::STAGE_BYTES;
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (CF::STAGES + s); };
    auto accf_bar = [&](int b) { return bar_base + 8u * (2 * CF::STAGES + b); };
    auto acce_bar = [&](int b) { return bar_base + 8u * (2 * CF::STAGES + 2 + b); };
    const uint32_t drain_bar = bar_base + 8u * (2 * CF::STAGES + 4);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(gbar + 8 * (2 * CF::STAGES + 5));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbar + 8 * (2 * CF::STAGES + 5) + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    WaitCtx w{abort_flag, dstate, limit_ns};

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), CF::EPI_WARPS);   // one arrive per epilogue warp
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), CF::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const int64_t num_units = src.num_units();

    auto producer_role = [&]() {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_mask = 0, last_parity = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                UnitInfo ui;
                src.unit(u, ui);
                const int y_a = (int)(ui.tm * BM), y_b = (int)(ui.tn * CF::BN);
                for (int kb = ui.kb0; kb < ui.kb1; ++kb) {
                    if (!wait_bounded(w, empty_bar(stage), phase ^ 1u, kSiteProducerEmpty)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(full_bar(stage), CF::STAGE_BYTES);
                    for (int t = 0; t < CF::A_PARTS; ++t)
                        tma_load_3d(a_smem + (stage * CF::A_PARTS + t) * CF::A_TILE, ui.ma,
                                    full_bar(stage), kb * CF::BK, y_a, t);
                    for (int t = 0; t < CF::B_PARTS; ++t)
                        tma_load_3d(b_smem + (stage * CF::B_PARTS + t) * CF::B_TILE, ui.mb,
                                    full_bar(stage), kb * CF::BK, y_b, t);
                    issued_mask |= 1u << stage;
                    last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == CF::STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            // Wait (bounded, even after an abort) for every copy still in flight.
            for (int s = 0; s < CF::STAGES; ++s) {
                if (!(issued_mask & (1u << s))) continue;
                const uint32_t par = (last_parity >> s) & 1u;
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(full_bar(s), par)) {
                    if (global_ns() - t0 > kDrainLimitNs) { record_timeout(w, kSiteDrain); break; }
                }
            }
        }
        __syncwarp();
    };
    auto mma_role = [&]() {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc = instr_desc<CF::FMT, CF::BN>();
            const uint64_t desc_a0 = smem_desc<RB>(a_smem), desc_b0 = smem_desc<RB>(b_smem);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            // One k-block: wait for its stage, issue every term pair's MMAs
            // into d_tmem, free the stage when they finish.
            auto kblock = [&](uint32_t d_tmem, uint32_t &accumulate) -> bool {
                if (!wait_bounded(w, full_bar(stage), phase, kSiteMmaFull)) return false;
                tc_fence_after();
                // The descriptor's start-address field is the byte address
                // >> 4, so offsetting a descriptor by whole 16-byte units
                // is an add: one base descriptor per stage and operand,
                // constant offsets for the term and the k-step.
                const uint64_t da = desc_a0 + (uint64_t)((stage * CF::A_PARTS * CF::A_TILE) >> 4);
                const uint64_t db = desc_b0 + (uint64_t)((stage * CF::B_PARTS * CF::B_TILE) >> 4);
#pragma unroll
                for (int q = 0; q < CF::NPAIRS; ++q) {
                    int sa, sb;
                    pair_of<MODE>(q, sa, sb);
#pragma unroll
                    for (int ks = 0; ks < CF::KSTEPS; ++ks) {
                        mma_issue<CF::TF32>(
                            d_tmem, da + (uint64_t)((sa * CF::A_TILE + ks * CF::KSTEP_BYTES) >> 4),
                            db + (uint64_t)((sb * CF::B_TILE + ks * CF::KSTEP_BYTES) >> 4), idesc,
                            accumulate);
                        accumulate = 1;
                    }
                }
                mma_commit(empty_bar(stage));     // frees the stage once these MMAs finish
                if (++stage == CF::STAGES) { stage = 0; phase ^= 1u; }
                return true;
            };
            if constexpr (CF::PROMO) {
                // Chunks of pk k-blocks, each into a fresh accumulator (the
                // two TMEM buffers alternate), handed to the epilogue warps
                // as soon as the chunk's MMAs finish.
                const int pk = src.chunk_kb;
                for (int64_t u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                    UnitInfo ui;
                    src.unit(u, ui);
                    int rel = 0;
                    uint32_t d_tmem = 0, accumulate = 0;
                    for (int kb = ui.kb0; kb < ui.kb1; ++kb) {
                        if (rel == 0) {
                            if (!wait_bounded(w, acce_bar(acc), acc_phase ^ 1u, kSiteMmaAccEmpty)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            d_tmem = tmem_base + (uint32_t)(acc * CF::BN);
                            accumulate = 0;
                        }
                        if (!kblock(d_tmem, accumulate)) { ok = false; break; }
                        if (++rel == pk || kb + 1 == ui.kb1) {
                            mma_commit(accf_bar(acc));    // chunk ready for the epilogue
                            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
                            rel = 0;
                        }
                    }
                }
            } else {
                for (int64_t u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                    if (!wait_bounded(w, acce_bar(acc), acc_phase ^ 1u, kSiteMmaAccEmpty)) break;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(acc * CF::BN);
                    uint32_t accumulate = 0;
                    UnitInfo ui;
                    src.unit(u, ui);
                    for (int kb = ui.kb0; kb < ui.kb1; ++kb) {
                        if (!kblock(d_tmem, accumulate)) { ok = false; break; }
                    }
                    if (!ok) break;
                    mma_commit(accf_bar(acc));            // accumulator ready for the epilogue
                    if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
                }
            }
            // Make sure no MMA is still running before TMEM is released.
            mma_commit(drain_bar);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(drain_bar, 0)) {
                if (global_ns() - t0 > kDrainLimitNs) { record_timeout(w, kSiteDrain); break; }
            }
        }
        __syncwarp();
    };
    auto promo_epilogue_role = [&]() {
      if constexpr (CF::PROMO) {
        // ------------- promoted epilogue (warps 4..11) -------------
        const int q = warp & 3;                       // TMEM lane quarter this warp may read
        const int hcol = ((warp - CF::EPI_WARP0) >> 2) * CF::ECOLS;   // first tile column
        const int pk = src.chunk_kb;
        int acc = 0;
        uint32_t acc_phase = 0;
        auto prefetch_unit = [&](int64_t v) {
            if (v >= num_units) return;
            UnitInfo pi;
            src.unit(v, pi);
            if (!pi.raw && pi.beta != 0.f)
                prefetch_tile_rows<CF::ECOLS>(pi.dst + hcol * pi.ldd, pi.ldd, pi.M,
                                              pi.N - hcol, pi.tm, pi.tn * (CF::BN / CF::ECOLS),
                                              q, lane);
        };
        prefetch_unit(blockIdx.x);
        bool ok = true;
        for (int64_t u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
            prefetch_unit(u + gridDim.x);
            int nch;
            {
                UnitInfo ui;
                src.unit(u, ui);
                const int nkb = ui.kb1 - ui.kb0;
                nch = nkb > 0 ? (nkb + pk - 1) / pk : 0;
            }
            float v[CF::ECOLS];
#pragma unroll
            for (int j = 0; j < CF::ECOLS; ++j) v[j] = 0.f;
            for (int ch = 0; ch < nch; ++ch) {
                // The TMEM loads are warp-collective: leave as a whole warp.
                const bool got = wait_bounded(w, accf_bar(acc), acc_phase, kSiteEpiAccFull);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) +
                                       (uint32_t)(acc * CF::BN + hcol);
                // 64 columns in flight per TMEM round trip (two per chunk):
                // the fold has to keep pace with the MMAs of the next chunk.
#pragma unroll
                for (int c = 0; c < CF::ECOLS; c += 64) {
                    uint32_t ra[16], rb[16], rc[16], rd[16];
                    tmem_ld16(taddr + (uint32_t)c, ra);
                    tmem_ld16(taddr + (uint32_t)(c + 16), rb);
                    tmem_ld16(taddr + (uint32_t)(c + 32), rc);
                    tmem_ld16(taddr + (uint32_t)(c + 48), rd);
                    tmem_wait64(ra, rb, rc, rd);
                    // the chunks are summed in order, each addition rounded
                    // to nearest (0 + x = x for the first)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[c + j] = __fadd_rn(v[c + j], __uint_as_float(ra[j]));
                        v[c + 16 + j] = __fadd_rn(v[c + 16 + j], __uint_as_float(rb[j]));
                        v[c + 32 + j] = __fadd_rn(v[c + 32 + j], __uint_as_float(rc[j]));
                        v[c + 48 + j] = __fadd_rn(v[c + 48 + j], __uint_as_float(rd[j]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce_bar(acc));
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            if (!ok) break;
            UnitInfo ui;            // looked up again: not kept live across the chunks
            src.unit(u, ui);
            float a = ui.raw ? 1.f : ui.alpha;
            if constexpr (MODE == 4) {
                // Undo the scaled split: the accumulator holds 2^(11 + e_i + f)
                // times the product (e_i the row's exponent, f the tile's
                // column block's). When a * 2^-(11 + e_i + f) is exact the
                // factor joins a (one rounding, as a * (v 2^-E) would give);
                // otherwise each value is scaled first, exactly unless it
                // leaves the FP32 range.
                static_assert(CF::BN == kFp16ColBlock, "one column block per tile");
                const int64_t row = ui.tm * BM + q * 32 + lane;
                const int ea = row < ui.M ? fp16_row_exp(src.amax[row], kFp16TopA) : 0;
                const int E = kFp16LoShift + ea + fp16_row_exp(src.bmax[ui.tn], kFp16TopB);
                if (pow2_scale_in_range(a, E)) {
                    a = scale_pow2(a, E);
                } else {
#pragma unroll
                    for (int j = 0; j < CF::ECOLS; ++j) v[j] = scale_pow2(v[j], E);
                }
            }
            store_regs<CF::BN, CF::ECOLS>(ui, v, hcol, q, lane, a);
        }
      }
    };
    auto epilogue_role = [&]() {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;                       // TMEM lane quarter this warp may read
        int acc = 0;
        uint32_t acc_phase = 0;
        // What a unit's epilogue will read (C when beta != 0, the factor's
        // array for the (1 - aux^2) epilogue) is requested from L2 one unit
        // ahead, while the tensor cores still work on it.
        auto prefetch_unit = [&](int64_t v) {
            if (v >= num_units) return;
            UnitInfo pi;
            src.unit(v, pi);
            if (!pi.raw && pi.beta != 0.f)
                prefetch_tile_rows<CF::BN>(pi.dst, pi.ldd, pi.M, pi.N, pi.tm, pi.tn, q, lane);
            if constexpr (Src::kEpi == 2)
                prefetch_tile_rows<CF::BN>(src.ep.aux, src.ep.ldaux, pi.M, pi.N, pi.tm, pi.tn, q,
                                           lane);
        };
        prefetch_unit(blockIdx.x);
        for (int64_t u = blockIdx.x; u < num_units; u += gridDim.x) {
            prefetch_unit(u + gridDim.x);
            // The TMEM loads below are warp-collective: leave (or stay) as a
            // whole warp even if only some lanes saw their wait expire.
            const bool got = wait_bounded(w, accf_bar(acc), acc_phase, kSiteEpiAccFull);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            UnitInfo ui;
            src.unit(u, ui);
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * CF::BN);
            if constexpr (Src::kEpi != 0)
                store_tile_epi<CF::BN, Src::kEpi>(ui, taddr, q, lane, src.ep);
            else
                store_tile<CF::BN, Src::kTri>(ui, taddr, q, lane);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(acc));
            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
        }
    };

    if constexpr (CF::PROMO) {
        // Registers move between whole warpgroups, so each setmaxnreg sits at
        // the top of a branch that a whole warpgroup takes.
        if (warp < 4) {
            asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(CF::REG_LOW));
            if (warp == 0) producer_role();
            else if (warp == 1) mma_role();
        } else {
            asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(CF::REG_HIGH));
            promo_epilogue_role();
        }
    } else {
        if (warp == 0) producer_role();
        else if (warp == 1) mma_role();
        else epilogue_role();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, CF::TMEM_COLS);
}

}  // namespace tcx
}  // namespace gb
