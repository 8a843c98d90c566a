// Split-precision SGEMM with the FP32 -> BF16 split fused into the
// tensor-core kernel: no separate pack pass and no workspace for operands.
//
// TMA brings FP32 tiles of the caller's A and B straight from their
// column-major storage into shared memory (a K-contiguous source as 128-byte
// rows with 128-byte swizzle, a rows-contiguous source as k-major rows
// without swizzle). Six converter warps read each tile, split every element
// into its BF16 terms (the same rounding as the pack pass, so results are
// bit-identical to the two-pass path) and write them, already transposed to
// K-major, into the 64-byte-swizzled layout tcgen05.mma reads. The MMA warp
// and the epilogue are those of the two-pass kernel. This is the paper's
// re-buffering of B' (Sec. 3) moved inside the kernel: the operands are
// re-laid out on their way from L2 to the tensor cores instead of in a
// separate pass through HBM.
//
// Pipelines (mbarrier handshakes, all waits bounded as in the two-pass
// kernel): TMA producer -> S1 FP32 stages -> converters -> S2 operand stages
// -> MMA warp -> 2 TMEM accumulators -> epilogue warps.
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2..5 epilogue,
// 6..11 converters (384 threads, one CTA per SM).
//
// Requirements (else the caller uses the two-pass path): A and B 16-byte
// aligned with leading dimensions that are multiples of 4 (TMA strides), a
// BF16 split algorithm, M, N, K < 2^31.
#include "f32_tile.cuh"

namespace gb {
namespace {

using namespace tcx;
using namespace fx;

constexpr int NCONV = 6;                      // converter warps
constexpr int CONV_WARP0 = 6;
constexpr int F_THREADS = (CONV_WARP0 + NCONV) * 32;

template <int MODE>                           // 1: BF16 x 2 terms, 2: BF16 x 3 terms
struct FCfg {
    static constexpr int PARTS = MODE == 2 ? 3 : 2;
    static constexpr int NPAIRS = MODE == 2 ? 6 : 3;
    static constexpr int BN = MODE == 2 ? 128 : 256;
    static constexpr int A_F32 = BM * FBK * 4;
    static constexpr int B_F32 = BN * FBK * 4;
    static constexpr int F32_BYTES = A_F32 + B_F32;
    static constexpr int A_OP = BM * 64;      // one term, 64-byte rows
    static constexpr int B_OP = BN * 64;
    static constexpr int OP_BYTES = PARTS * (A_OP + B_OP);
    // One ring of stages: TMA writes the FP32 tiles, the converters turn them
    // into the BF16 terms in place (the terms overwrite the FP32 bytes), the
    // MMAs read the terms, and the stage goes back to the producer.
    static constexpr int STAGE = F32_BYTES > OP_BYTES ? F32_BYTES : OP_BYTES;
    static constexpr int STAGES = 4;
    static constexpr int ITEMS_A = (BM * 4 + NCONV * 32 - 1) / (NCONV * 32);
    static constexpr int ITEMS_B = (BN * 4 + NCONV * 32 - 1) / (NCONV * 32);
    static constexpr int TMEM_COLS = 2 * BN;
    static constexpr int NBARS = 3 * STAGES + 5;
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE + 8 * NBARS + 16;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
    static_assert(STAGE % 1024 == 0 && A_F32 % 1024 == 0, "tile alignment");
};

// AND of `pred` over the converter threads, which also synchronises them
// (named barrier 2; barrier 0 is __syncthreads).
__device__ __forceinline__ bool conv_all(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, 2, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(NCONV * 32)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void conv_sync() {
    asm volatile("bar.sync 2, %0;" ::"n"(NCONV * 32) : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(F_THREADS, 1)
tc_fused_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                int akc, int bkc, int64_t M, int64_t N, int64_t K, float alpha, float beta,
                float *__restrict__ C, int64_t ldc, float *__restrict__ part, int splits,
                DeviceState *dstate, uint64_t limit_ns) {
    using CF = FCfg<MODE>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    // stage s at base + s*STAGE: FP32 A tile at +0, FP32 B tile at +A_F32;
    // after conversion, A terms at +p*A_OP and B terms at +PARTS*A_OP + p*B_OP
    const uint32_t bar_base = base + CF::STAGES * CF::STAGE;
    uint8_t *gbar = gbase + CF::STAGES * CF::STAGE;
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto conv_bar = [&](int s) { return bar_base + 8u * (CF::STAGES + s); };
    auto empty_bar = [&](int s) { return bar_base + 8u * (2 * CF::STAGES + s); };
    auto accf_bar = [&](int b) { return bar_base + 8u * (3 * CF::STAGES + b); };
    auto acce_bar = [&](int b) { return bar_base + 8u * (3 * CF::STAGES + 2 + b); };
    const uint32_t drain_bar = bar_base + 8u * (3 * CF::STAGES + 4);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(gbar + 8 * CF::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbar + 8 * CF::NBARS + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    WaitCtx w{abort_flag, dstate, limit_ns};

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(conv_bar(s), NCONV);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 4);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_tmap(&mapA);
        prefetch_tmap(&mapB);
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), CF::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    SingleSource<CF::BN, FBK> src;
    src.ma = &mapA; src.mb = &mapB;
    src.M = M; src.N = N; src.K = K;
    src.alpha = alpha; src.beta = beta;
    src.C = C; src.ldc = ldc;
    src.part = part; src.splits = splits;
    src.tiles_m = (int)((M + BM - 1) / BM);
    src.tiles_n = (int)((N + CF::BN - 1) / CF::BN);
    src.nkb = (int)((K + FBK - 1) / FBK);
    const int64_t num_units = src.num_units();

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (FP32 tiles) ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_mask = 0, last_parity = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                UnitInfo ui;
                src.unit(u, ui);
                const int ra = (int)(ui.tm * BM), rb = (int)(ui.tn * CF::BN);
                for (int kb = ui.kb0; kb < ui.kb1; ++kb) {
                    if (!wait_bounded(w, empty_bar(stage), phase ^ 1u, kSiteProducerEmpty)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fa = base + stage * CF::STAGE;
                    mbar_arrive_expect_tx(full_bar(stage), CF::F32_BYTES);
                    // K-contiguous source: (x = k, y = row); else (x = row, y = k)
                    if (akc) tma_load_2d(fa, &mapA, full_bar(stage), kb * FBK, ra);
                    else     tma_load_2d(fa, &mapA, full_bar(stage), ra, kb * FBK);
                    if (bkc) tma_load_2d(fa + CF::A_F32, &mapB, full_bar(stage), kb * FBK, rb);
                    else     tma_load_2d(fa + CF::A_F32, &mapB, full_bar(stage), rb, kb * FBK);
                    issued_mask |= 1u << stage;
                    last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == CF::STAGES) { stage = 0; phase ^= 1u; }
                }
            }
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
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc = instr_desc<kFmtBF16, CF::BN>();
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < num_units && ok; u += gridDim.x) {
                if (!wait_bounded(w, acce_bar(acc), acc_phase ^ 1u, kSiteMmaAccEmpty)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * CF::BN);
                uint32_t accumulate = 0;
                UnitInfo ui;
                src.unit(u, ui);
                for (int kb = ui.kb0; kb < ui.kb1; ++kb) {
                    if (!wait_bounded(w, conv_bar(stage), phase, kSiteMmaFull)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = base + stage * CF::STAGE;
#pragma unroll
                    for (int q = 0; q < CF::NPAIRS; ++q) {
                        int sa, sbt;
                        pair_of<MODE>(q, sa, sbt);
                        const uint32_t a0 = sb + sa * CF::A_OP;
                        const uint32_t b0 = sb + CF::PARTS * CF::A_OP + sbt * CF::B_OP;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            mma_issue<false>(d_tmem, smem_desc<64>(a0 + ks * 32),
                                             smem_desc<64>(b0 + ks * 32), idesc, accumulate);
                            accumulate = 1;
                        }
                    }
                    mma_commit(empty_bar(stage));      // stage back to the producer
                    if (++stage == CF::STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(accf_bar(acc));
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            mma_commit(drain_bar);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(drain_bar, 0)) {
                if (global_ns() - t0 > kDrainLimitNs) { record_timeout(w, kSiteDrain); break; }
            }
        }
        __syncwarp();
    } else if (warp < CONV_WARP0) {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int64_t u = blockIdx.x; u < num_units; u += gridDim.x) {
            const bool got = wait_bounded(w, accf_bar(acc), acc_phase, kSiteEpiAccFull);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            UnitInfo ui;
            src.unit(u, ui);
            store_tile<CF::BN>(ui, tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * CF::BN),
                               q, lane);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(acc));
            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
        }
    } else {
        // ---------------- converters (warps 6..11) ----------------
        // Per stage: read the whole FP32 tile into registers, synchronise
        // the converter warps (the terms overwrite the FP32 bytes), split and
        // write the terms, make them visible to the tensor cores, signal.
        const int ct = threadIdx.x - CONV_WARP0 * 32;
        int stage = 0;
        uint32_t phase = 0;
        for (int64_t u = blockIdx.x; u < num_units; u += gridDim.x) {
            UnitInfo ui;
            src.unit(u, ui);
            bool ok = true;
            for (int kb = ui.kb0; kb < ui.kb1; ++kb) {
                // every converter thread waits; all leave or all stay
                if (!conv_all(wait_bounded(w, full_bar(stage), phase, kSiteConvert))) {
                    ok = false;
                    break;
                }
                uint8_t *sp = gbase + stage * CF::STAGE;
                const float *fa = reinterpret_cast<const float *>(sp);
                const float *fb = reinterpret_cast<const float *>(sp + CF::A_F32);
                float va[CF::ITEMS_A][8], vb[CF::ITEMS_B][8];
#pragma unroll
                for (int j = 0; j < CF::ITEMS_A; ++j) {
                    const int i = ct + j * NCONV * 32;
                    if (i < BM * 4) read8<BM>(fa, akc != 0, i % BM, i / BM, va[j]);
                }
#pragma unroll
                for (int j = 0; j < CF::ITEMS_B; ++j) {
                    const int i = ct + j * NCONV * 32;
                    if (i < CF::BN * 4) read8<CF::BN>(fb, bkc != 0, i % CF::BN, i / CF::BN, vb[j]);
                }
                conv_sync();                           // all FP32 reads done before any term write
#pragma unroll
                for (int j = 0; j < CF::ITEMS_A; ++j) {
                    const int i = ct + j * NCONV * 32;
                    if (i < BM * 4) write8<CF::PARTS>(sp, CF::A_OP, i % BM, i / BM, va[j]);
                }
#pragma unroll
                for (int j = 0; j < CF::ITEMS_B; ++j) {
                    const int i = ct + j * NCONV * 32;
                    if (i < CF::BN * 4)
                        write8<CF::PARTS>(sp + CF::PARTS * CF::A_OP, CF::B_OP, i % CF::BN, i / CF::BN, vb[j]);
                }
                fence_async_shared();                  // term writes -> tensor-core reads
                __syncwarp();
                if (lane == 0) mbar_arrive(conv_bar(stage));
                if (++stage == CF::STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, CF::TMEM_COLS);
}

template <int MODE>
cudaError_t launch_fused_mode(const FusedArgs &a, cudaStream_t s) {
    using CF = FCfg<MODE>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_fused_kernel<MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    // op(A)[i,p]: stored A is K-contiguous iff transposed (stored K x M);
    // op(B)^T[j,p]: stored B is K-contiguous iff not transposed (stored K x N).
    const bool akc = a.ta, bkc = !a.tb;
    alignas(64) CUtensorMap ma, mb;
    if (!make_f32_map(&ma, a.A, akc ? a.k : a.m, akc ? a.m : a.k, a.lda, akc, BM) ||
        !make_f32_map(&mb, a.B, bkc ? a.k : a.n, bkc ? a.n : a.k, a.ldb, bkc, CF::BN))
        return cudaErrorNotSupported;
    const int splits = a.part ? (a.splits > 1 ? a.splits : 1) : 1;
    const int64_t units = ((a.m + BM - 1) / BM) * ((a.n + CF::BN - 1) / CF::BN) * splits;
    if (units > 2147483647LL) return cudaErrorNotSupported;
    int grid = a.sm_count > 0 ? a.sm_count : 1;
    if (units < grid) grid = (int)units;
    tc_fused_kernel<MODE><<<grid, F_THREADS, CF::SMEM_BYTES, s>>>(
        ma, mb, akc ? 1 : 0, bkc ? 1 : 0, a.m, a.n, a.k, a.alpha, a.beta, a.C, a.ldc,
        splits > 1 ? a.part : nullptr, splits, a.dstate, (uint64_t)a.wait_limit * 1000ull);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    return launch_splitk_reduce(a.m, a.n, splits, a.part, a.alpha, a.beta, a.C, a.ldc, s);
}

}  // namespace

bool fused_supported(int mode, const float *A, int64_t lda, const float *B, int64_t ldb, int64_t m,
                     int64_t n, int64_t k) {
    if (mode != 1 && mode != 2) return false;
    if (!f32_tma_ok(A, lda) || !f32_tma_ok(B, ldb)) return false;
    return m < 2147483647LL && n < 2147483647LL && k < 2147483647LL;
}

cudaError_t launch_tc_fused(const FusedArgs &a, cudaStream_t s) {
    switch (a.mode) {
        case 1: return launch_fused_mode<1>(a, s);
        case 2: return launch_fused_mode<2>(a, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace gb
