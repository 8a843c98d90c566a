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

__device__ __noinline__ void record_timeout(const WaitCtx &w, int site) {
    atomicCAS(&w.dstate->err[0], 0u, (unsigned)site);
    atomicAdd(&w.dstate->err[1], 1u);
    *w.abort = 1;
}

// Bounded wait for the phase of `bar` with the given parity to complete.
// Returns false if the limit expired (recorded) or another role aborted.
__device__ __forceinline__ bool wait_bounded(const WaitCtx &w, uint32_t bar, uint32_t parity,
                                             int site) {
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

// Instruction descriptor (kind::f16 / kind::tf32): D format F32 (bits 4-5 =
// 1), A and B formats (bits 7-9, 10-12: 1 = BF16, 2 = TF32), both K-major
// (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <bool TF32, int N, int M = BM>
__device__ __forceinline__ constexpr uint32_t instr_desc() {
    constexpr uint32_t fmt = TF32 ? 2u : 1u;
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




// Term pair (A term, B term) for step q, smallest weight first.
template <int MODE>
__device__ __forceinline__ void pair_of(int q, int &sa, int &sb) {
    if (MODE == 2) {
        const int a[6] = {0, 1, 2, 0, 1, 0};
        const int b[6] = {2, 1, 0, 1, 0, 0};
        sa = a[q]; sb = b[q];
    } else {
        const int a[3] = {1, 0, 0};
        const int b[3] = {0, 1, 0};
        sa = a[q]; sb = b[q];
    }
}

// Tile raster in groups of GROUP_M tile rows (32-bit: the host guarantees
// that the number of work units fits in an int).

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

}  // namespace tcx
}  // namespace gb
