// PTX helpers shared by the tensor-core kernels (tcgen05, TMEM, TMA,
// mbarrier) and the bounded-wait machinery. Included by one translation unit
// per kernel family; everything here is internal to the library.
#pragma once

#include "internal.h"

namespace gb {
namespace tcx {

constexpr int BM = 128;                        // MMA M (rows of a tile, TMEM lanes)
// Limit for the final drains of in-flight copies and MMAs. These always
// complete in hardware within microseconds; the generous fixed limit keeps
// the CTA from exiting with asynchronous work outstanding even when the
// caller set a very short limit for the ordinary waits.
constexpr uint64_t kDrainLimitNs = 4000000000ull;

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct WaitCtx {
    volatile int *abort;          // CTA-wide abort flag (shared memory)
    DeviceState *dstate;          // handle's device error word
    uint64_t limit_ns;
};

static __device__ __noinline__ void record_timeout(const WaitCtx &w, int site) {
    atomicCAS(&w.dstate->err[0], 0u, (unsigned)site);
    atomicAdd(&w.dstate->err[1], 1u);
    *w.abort = 1;
}

// Bounded wait for the phase of `bar` with the given parity to complete.
// Returns false if the limit expired (recorded) or another role aborted.
__device__ __forceinline__ bool wait_bounded(const WaitCtx &w, uint32_t bar, uint32_t parity,
                                             int site) {
    // (A variant that sleeps in try_wait with a suspend-time hint measured
    // slower on short-K shapes: the wake-up latency lands on every tile
    // hand-off. Plain polling it is.)
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*w.abort) return false;
        if ((it & 15u) == 15u && global_ns() - t0 > w.limit_ns) {
            record_timeout(w, site);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile written by TMA
// with an RB-byte swizzle (RB = 128 or 64): rows of RB bytes, 8-row swizzle
// atoms (8*RB bytes) stacked along M/N. Fields: start address >> 4 (bits
// 0-13), leading byte offset >> 4 (16-29; unused for swizzled K-major, set to
// 1), stride byte offset >> 4 (32-45; 8*RB bytes between 8-row groups),
// descriptor version 1 (46-47), base offset 0 (49-51; atoms are aligned),
// layout type (61-63): 2 = 128-byte swizzle, 4 = 64-byte swizzle.
template <int RB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    static_assert(RB == 128 || RB == 64, "row bytes");
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8 * RB) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(RB == 128 ? 2 : 4) << 61;
    return d;
}

// Operand formats of the instruction descriptor (A and B alike).
enum : int { kFmtF16 = 0, kFmtBF16 = 1, kFmtTF32 = 2 };

// Instruction descriptor (kind::f16 / kind::tf32): D format F32 (bits 4-5 =
// 1), A and B formats (bits 7-9, 10-12: 0 = F16, 1 = BF16, 2 = TF32), both
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int FMT, int N, int M = BM>
__device__ __forceinline__ constexpr uint32_t instr_desc() {
    constexpr uint32_t fmt = (uint32_t)FMT;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    if (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns: thread t of the warp gets
// row (lane base + t), columns col..col+15. The load is asynchronous: the
// registers are valid only after tmem_wait().
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Waits for this thread's outstanding TMEM loads. The 16 registers of the
// load are in/out operands, so the compiler cannot move any use of them
// above the wait (the load writes them asynchronously).
__device__ __forceinline__ void tmem_wait16(uint32_t r[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

// Waits for this thread's outstanding TMEM loads, with the 32 registers of
// two 16-column loads as in/out operands (see tmem_wait16).
__device__ __forceinline__ void tmem_wait32(uint32_t a[16], uint32_t b[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                   "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]),
                   "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]),
                   "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                   "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]),
                   "+r"(b[14]), "+r"(b[15])
                 :
                 : "memory");
}

// Waits for this thread's outstanding TMEM loads, with the 48 registers of
// three 16-column loads as in/out operands (see tmem_wait16).
__device__ __forceinline__ void tmem_wait48(uint32_t a[16], uint32_t b[16], uint32_t c[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]), "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7]), "+r"(c[8]), "+r"(c[9]), "+r"(c[10]), "+r"(c[11]), "+r"(c[12]), "+r"(c[13]), "+r"(c[14]), "+r"(c[15])
                 :
                 : "memory");
}

// Waits for this thread's outstanding TMEM loads, with the 64 registers of
// four 16-column loads as in/out operands (see tmem_wait16).
__device__ __forceinline__ void tmem_wait64(uint32_t a[16], uint32_t b[16], uint32_t c[16],
                                            uint32_t d[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]), "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7]), "+r"(c[8]), "+r"(c[9]), "+r"(c[10]), "+r"(c[11]), "+r"(c[12]), "+r"(c[13]), "+r"(c[14]), "+r"(c[15]), "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7]), "+r"(d[8]), "+r"(d[9]), "+r"(d[10]), "+r"(d[11]), "+r"(d[12]), "+r"(d[13]), "+r"(d[14]), "+r"(d[15])
                 :
                 : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns from this thread's registers:
// thread t of the warp writes row (lane base + t). Asynchronous: complete
// only after tmem_wait_st().
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t r[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D (+)= A * B with the A operand in tensor memory (128 lanes = M rows, K
// packed two 16-bit values per 32-bit column starting at a_tmem, the lower
// K in the low half) and B in shared memory (descriptor), kind::f16.
__device__ __forceinline__ void mma_issue_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Term pair (A term, B term) for step q, smallest weight first.
template <int MODE>
__device__ __forceinline__ void pair_of(int q, int &sa, int &sb) {
    if (MODE == 4) {
        // scaled FP16: A terms (2^11 h, h, l), B terms (h, l); the products
        // h_a l_b, l_a h_b and 2^11 h_a h_b, so that one accumulator holds
        // 2^11 (h_a h_b + (h_a l_b + l_a h_b) 2^-11)
        const int a[3] = {1, 2, 0};
        const int b[3] = {1, 0, 0};
        sa = a[q]; sb = b[q];
    } else if (MODE == 3) {
        // all nine products, by weight: 2^-32, 2^-24 (x2), 2^-16 (x3), 2^-8 (x2), 1
        const int a[9] = {2, 1, 2, 0, 1, 2, 0, 1, 0};
        const int b[9] = {2, 2, 1, 2, 1, 0, 1, 0, 0};
        sa = a[q]; sb = b[q];
    } else if (MODE == 2) {
        const int a[6] = {0, 1, 2, 0, 1, 0};
        const int b[6] = {2, 1, 0, 1, 0, 0};
        sa = a[q]; sb = b[q];
    } else {
        const int a[3] = {1, 0, 0};
        const int b[3] = {0, 1, 0};
        sa = a[q]; sb = b[q];
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Makes this thread's generic-proxy shared-memory writes visible to the
// async proxy (tensor-core operand reads).
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


constexpr int GROUP_M = 16;                    // tile raster: 16 M-tiles per group

// Tile raster in groups of GROUP_M tile rows (32-bit: the host guarantees
// that the number of work units fits in an int).
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int64_t &tm,
                                            int64_t &tn) {
    const int per_group = GROUP_M * tiles_n;
    const int g = tile / per_group;
    const int first_m = g * GROUP_M;
    const int gm = (tiles_m - first_m) < GROUP_M ? (tiles_m - first_m) : GROUP_M;
    const int r = tile - g * per_group;
    tm = first_m + r % gm;
    tn = r / gm;
}

// What one work unit is: the operands' tensor maps, the output tile, the
// range of k-blocks, and where and how the result is written.
struct UnitInfo {
    const CUtensorMap *ma, *mb;
    int64_t M, N;                 // the problem's output size
    int64_t tm, tn;               // tile coordinates
    int kb0, kb1;                 // k-blocks [kb0, kb1)
    float alpha, beta;
    float *dst;                   // C, or this slice's partial-sum buffer
    int64_t ldd;
    bool raw;                     // write raw sums (split-K partial), no alpha/beta
    bool lower;                   // triangle sources: keep col <= row (else col >= row)
};

// Asks L2 for the part of a column-major M x N array (leading dimension ld)
// that epilogue warp q will read for tile (tm, tn): rows tm*128 + 32q ..
// +31 of the tile's columns, 128 contiguous bytes per column (two lines when
// they straddle a line boundary). Issued before the tile's accumulator is
// ready, so that the epilogue's reads of it come from L2, not DRAM.
__device__ __forceinline__ void prefetch_l2(const float *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int BN>
__device__ __forceinline__ void prefetch_tile_rows(const float *base, int64_t ld, int64_t M,
                                                   int64_t N, int64_t tm, int64_t tn, int q,
                                                   int lane) {
    const int64_t r0 = tm * BM + q * 32;
    if (r0 >= M) return;
    const int64_t last = (M - 1 - r0 < 31 ? M - 1 - r0 : 31);
    const int64_t c0 = tn * BN;
#pragma unroll 1
    for (int c = lane; c < BN && c0 + c < N; c += 32) {
        const float *col = base + r0 + (c0 + c) * ld;
        prefetch_l2(col);
        prefetch_l2(col + last);
    }
}

// One GEMM: units are (tile, K slice) pairs in the grouped raster order.
// Split units write raw partial sums to `part` (slice s at part + s*M*N,
// column-major, ld = M); a separate pass reduces them.
template <int BN, int BK, int EPI = 0>
struct SingleSource {
    static constexpr bool kTri = false;
    static constexpr int kEpi = EPI;
    EpiOp ep;                     // the fused elementwise operation (EPI != 0)
    const CUtensorMap *ma, *mb;
    int64_t M, N, K;
    float alpha, beta;
    float *C;
    int64_t ldc;
    float *part;
    int splits;
    int tiles_m, tiles_n;
    int nkb;
    int chunk_kb;                 // promoted accumulation: k-blocks per chunk
    const uint32_t *amax, *bmax;  // scaled FP16 split: row / column maxima (FP32 bits)
    __device__ __forceinline__ int64_t num_units() const {
        return (int64_t)tiles_m * tiles_n * splits;
    }
    __device__ __forceinline__ void unit(int64_t u64, UnitInfo &ui) const {
        const int u = (int)u64;
        tile_coords(u / splits, tiles_m, tiles_n, ui.tm, ui.tn);
        const int sl = u % splits;
        ui.kb0 = (int)((int64_t)sl * nkb / splits);
        ui.kb1 = (int)((int64_t)(sl + 1) * nkb / splits);
        ui.ma = ma; ui.mb = mb;
        ui.M = M; ui.N = N;
        ui.alpha = alpha; ui.beta = beta;
        ui.raw = part != nullptr;
        ui.dst = part ? part + sl * M * N : C;
        ui.ldd = part ? M : ldc;
    }
};

// Epilogue of one work unit for one epilogue warp: TMEM lanes q*32..q*32+31
// (rows of the tile) of the accumulator at TMEM address `taddr`, BN columns,
// to C (alpha/beta) or to a split-K partial buffer (raw sums). TRI: only the
// elements of the ui.lower (col <= row) or upper (col >= row) triangle are
// stored (and C is read only there).
template <int BN, bool TRI = false>
__device__ __forceinline__ void store_tile(const UnitInfo &ui, uint32_t taddr, int q, int lane) {
    const int64_t M = ui.M, N = ui.N, ldd = ui.ldd;
    float *dst = ui.dst;
    const float alpha = ui.alpha, beta = ui.beta;
    const bool part = ui.raw;
    const bool empty = ui.kb0 >= ui.kb1;   // an empty K range contributes 0 (TMEM unwritten)
    const float a = part ? 1.f : alpha;
    const int64_t row = ui.tm * BM + q * 32 + lane;
    const int64_t col0 = ui.tn * BN;
    const bool row_ok = row < M;
    // Chunks of 16 columns: load from TMEM, wait, store; a warp writes
    // 128 contiguous bytes of one column per store instruction. (Keeping
    // more TMEM loads in flight, pipelining them against the stores, or
    // staging whole 512-byte columns through shared memory all measured
    // slower on the store-bound K = 64 shapes.) Interior tiles take a
    // path with no per-element checks and a pointer bump per column:
    // on store-bound shapes the epilogue's instruction count is the limit.
    bool interior = (ui.tm * BM + BM <= M) && (col0 + BN <= N);
    if (TRI)   // the whole tile inside the triangle
        interior = interior && (ui.lower ? col0 + BN - 1 <= ui.tm * BM : col0 >= ui.tm * BM + BM - 1);
    float *colp = dst + row + col0 * ldd;
    if (interior && !part && beta != 0.f) {
        // C of the next 16 columns is requested before this chunk's TMEM
        // wait and stores, so its latency overlaps them: one memory round
        // trip per tile instead of one per chunk. (Every load of a chunk is
        // issued before the previous chunk's stores, which a store could
        // otherwise alias.)
        float cv[16];
        {
            const float *qc = colp;
#pragma unroll
            for (int j = 0; j < 16; ++j) { cv[j] = *qc; qc += ldd; }
        }
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            uint32_t r[16];
            tmem_ld16(taddr + (uint32_t)c, r);
            float cn[16];
            if (c + 16 < BN) {
                const float *qn = colp + (c + 16) * ldd;
#pragma unroll
                for (int j = 0; j < 16; ++j) { cn[j] = *qn; qn += ldd; }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) cn[j] = 0.f;
            }
            tmem_wait16(r);
            if (empty) {
#pragma unroll
                for (int j = 0; j < 16; ++j) r[j] = 0u;
            }
            float *p = colp + c * ldd;
#pragma unroll
            for (int j = 0; j < 16; ++j) { *p = fmaf(a, __uint_as_float(r[j]), beta * cv[j]); p += ldd; }
#pragma unroll
            for (int j = 0; j < 16; ++j) cv[j] = cn[j];
        }
        return;
    }
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
        uint32_t r[16];
        tmem_ld16(taddr + (uint32_t)c, r);
        tmem_wait16(r);
        if (empty) {
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = 0u;
        }
        float *p = colp + c * ldd;
        if (interior) {
            if (part || beta == 0.f) {
#pragma unroll
                for (int j = 0; j < 16; ++j) { *p = a * __uint_as_float(r[j]); p += ldd; }
            } else {
                // all 16 C values are read before the first store: a store
                // may alias a later load, and interleaving them would
                // serialise 16 memory latencies
                float cv[16];
                const float *qc = p;
#pragma unroll
                for (int j = 0; j < 16; ++j) { cv[j] = *qc; qc += ldd; }
#pragma unroll
                for (int j = 0; j < 16; ++j) { *p = fmaf(a, __uint_as_float(r[j]), beta * cv[j]); p += ldd; }
            }
            continue;
        }
        if (!row_ok) continue;
        int jlo = 0, jhi = (int)(N - (col0 + c) < 16 ? N - (col0 + c) : 16);
        if (TRI) {   // columns col0 + c + j inside the triangle
            const int64_t d = row - (col0 + c);
            if (ui.lower) jhi = d + 1 < jhi ? (int)(d + 1 < 0 ? 0 : d + 1) : jhi;
            else jlo = d > 0 ? (int)(d < 16 ? d : 16) : 0;
        }
        const bool rd = !part && beta != 0.f;
        float cv[16];
        const float *qc = p;
#pragma unroll
        for (int j = 0; j < 16; ++j) { cv[j] = (rd && j >= jlo && j < jhi) ? *qc : 0.f; qc += ldd; }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j >= jlo && j < jhi)
                *p = rd ? fmaf(a, __uint_as_float(r[j]), beta * cv[j]) : a * __uint_as_float(r[j]);
            p += ldd;
        }
    }
}

// Epilogue with a fused elementwise operation (EPI = EpiOp::kind, see
// internal.h) after v = alpha*acc + beta*C; whole-K results only (no
// split-K). The operations round exactly as the separate passes would:
// kind 1 adds the bias in FP32 then applies tanhf; kind 2 multiplies by
// fmaf(-h, h, 1).
template <int BN, int EPI>
__device__ __forceinline__ void store_tile_epi(const UnitInfo &ui, uint32_t taddr, int q, int lane,
                                               const EpiOp &ep) {
    const int64_t M = ui.M, N = ui.N, ldd = ui.ldd;
    const float alpha = ui.alpha, beta = ui.beta;
    const bool empty = ui.kb0 >= ui.kb1;
    const int64_t row = ui.tm * BM + q * 32 + lane;
    const int64_t col0 = ui.tn * BN;
    const bool row_ok = row < M;
    const bool rd = beta != 0.f;
    const float bias = (EPI == 1 && row_ok) ? ep.bias[row] : 0.f;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
        uint32_t r[16];
        tmem_ld16(taddr + (uint32_t)c, r);
        tmem_wait16(r);
        if (!row_ok) continue;
        const int ncol = (int)(N - (col0 + c) < 16 ? N - (col0 + c) : 16);
        float *p = ui.dst + row + (col0 + c) * ldd;
        const float *ax = EPI == 2 ? ep.aux + row + (col0 + c) * ep.ldaux : nullptr;
        float cv[16], hv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            cv[j] = (rd && j < ncol) ? p[j * ldd] : 0.f;
            hv[j] = (EPI == 2 && j < ncol) ? ax[j * ep.ldaux] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j >= ncol) continue;
            const float acc = empty ? 0.f : __uint_as_float(r[j]);
            float v = rd ? fmaf(alpha, acc, beta * cv[j]) : alpha * acc;
            if (EPI == 1) {
                v = v + bias;
                if (ep.tanh_act) v = tanhf(v);
            } else if (EPI == 2) {
                v = v * fmaf(-hv[j], hv[j], 1.f);
            }
            p[j * ldd] = v;
        }
    }
}

}  // namespace tcx
}  // namespace gb
