// Split-precision SGEMM on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
// Input: the split/pack pass has written every FP32 element of op(A) and of
// op(B)^T as 2 or 3 lower-precision terms (TF32 or BF16), each term as a
// K-contiguous [rows][kpad] array. This kernel forms
//     acc = sum over term pairs (s, t) of  A_s * B_t^T      (FP32 in TMEM)
//     C   = alpha * acc + beta * C                           (fused epilogue)
// with the pairs ordered smallest weight first:
//   2 terms (h, l):      l*h, h*l, h*h
//   3 terms (h, m, l):   h*l, m*m, l*h, h*m, m*h, h*h
// Dropping l*l (and the 2^-24-weight pairs for 3 terms) keeps the error of
// every product near FP32 round-off, which is how the split recovers FP32
// accuracy from BF16/TF32 multipliers.
//
// The paper's Emmerald organises SGEMM around keeping operands close to the
// arithmetic units: a register-resident block of C, a k-block of A and B
// staged in L1, prefetch of the next block, and L2 blocking (Sec. 2, 3).
// On sm_103a the same roles are:
//   * C block in registers  -> a 128 x BN FP32 accumulator in tensor memory
//     (TMEM), two of them so the epilogue of one tile overlaps the next;
//   * L1 staging + prefetch -> a ring of shared-memory stages filled by TMA
//     (cp.async.bulk.tensor) ahead of the MMAs, handshaken with mbarriers:
//     64-byte rows (64-byte swizzle) in four 48 KiB stages for two terms or
//     three 72 KiB stages for three, or 128-byte rows (128-byte swizzle) in
//     two 96 KiB stages for the shapes tc_rb128() picks (K <= 128, short
//     3-term GEMMs with few tiles);
//   * the inner loop        -> tcgen05.mma (M = 128, N = BN, K = 16 BF16 or
//     8 TF32 per instruction) issued by one thread;
//   * L2 blocking           -> a persistent grid (one CTA per SM; two with the
//     grouped kernel's smaller configuration) walking the output tiles in
//     groups of 16 M-tiles so concurrently running CTAs share A and B panels
//     in L2.
// Warp roles in a 192-thread CTA: warp 0 = TMA producer, warp 1 = TMEM owner
// and MMA issuer, warps 2..5 = epilogue (TMEM -> registers -> global).
//
// Every mbarrier wait is bounded by a wall-clock limit (globaltimer). On
// expiry the thread records the wait site in the handle's device error word,
// raises a CTA-wide abort flag that every other wait also polls, and all
// roles leave their loops; the producer then waits (bounded) for its
// in-flight copies, the MMA issuer for its in-flight MMAs, and TMEM is freed
// before the CTA exits. No trap, no unbounded spin.
#include <cudaTypedefs.h>
#include <stdlib.h>

#include "tc_body.cuh"

namespace gb {
namespace {

using namespace tcx;
template <int MODE, int RB, int EPI>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_sgemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                int64_t M, int64_t N, int64_t K, float alpha, float beta, float *__restrict__ C,
                int64_t ldc, float *__restrict__ part, int splits, DeviceState *dstate,
                uint64_t limit_ns, EpiOp ep) {
    using CF = Cfg<MODE, RB>;
    if (threadIdx.x == 0) {
        prefetch_tmap(&mapA);
        prefetch_tmap(&mapB);
    }
    SingleSource<CF::BN, CF::BK, EPI> src;
    src.ep = ep;
    src.ma = &mapA; src.mb = &mapB;
    src.M = M; src.N = N; src.K = K;
    src.alpha = alpha; src.beta = beta;
    src.C = C; src.ldc = ldc;
    src.part = part; src.splits = splits;
    src.tiles_m = (int)((M + BM - 1) / BM);
    src.tiles_n = (int)((N + CF::BN - 1) / CF::BN);
    src.nkb = (int)((K + CF::BK - 1) / CF::BK);
    tc_body<MODE, RB>(src, dstate, limit_ns);
}

// Promoted accumulation: fresh FP32 accumulator every chunk_kb k-blocks,
// chunks added in FP32 round-to-nearest by eight epilogue warps.
template <int MODE>
__global__ void __launch_bounds__(PromoCfg<MODE>::THREADS, 1)
tc_promo_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                int64_t M, int64_t N, int64_t K, float alpha, float beta, float *__restrict__ C,
                int64_t ldc, float *__restrict__ part, int splits, int chunk_kb,
                const uint32_t *amax, const uint32_t *bmax, DeviceState *dstate,
                uint64_t limit_ns) {
    using CF = PromoCfg<MODE>;
    if (threadIdx.x == 0) {
        prefetch_tmap(&mapA);
        prefetch_tmap(&mapB);
    }
    SingleSource<CF::BN, CF::BK, 0> src;
    src.ma = &mapA; src.mb = &mapB;
    src.M = M; src.N = N; src.K = K;
    src.alpha = alpha; src.beta = beta;
    src.C = C; src.ldc = ldc;
    src.part = part; src.splits = splits;
    src.tiles_m = (int)((M + BM - 1) / BM);
    src.tiles_n = (int)((N + CF::BN - 1) / CF::BN);
    src.nkb = (int)((K + CF::BK - 1) / CF::BK);
    src.chunk_kb = chunk_kb;
    src.amax = amax; src.bmax = bmax;
    tc_body<MODE, CF::ROW_BYTES, SingleSource<CF::BN, CF::BK, 0>, CF>(src, dstate, limit_ns);
}

template <int MODE, int V>
__global__ void __launch_bounds__(NUM_THREADS, GroupedCfgV<MODE, V>::CTAS)
tc_grouped_kernel(const TcProblem *__restrict__ probs, const TcItem *__restrict__ items,
                  int64_t nitems, DeviceState *dstate, uint64_t limit_ns) {
    using CF = GroupedCfgV<MODE, V>;
    GroupSource<CF::BN, CF::BK> src{probs, items, nitems};
    tc_body<MODE, CF::ROW_BYTES, GroupSource<CF::BN, CF::BK>, CF>(src, dstate, limit_ns);
}

// C = alpha * (sum over slices s = 0..S-1, in that order, of part_s) + beta*C
// (C not read when beta == 0). part_s is column-major M x N with ld = M.
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int S, const float *__restrict__ part,
                                     float alpha, float beta, float *__restrict__ C, int64_t ldc) {
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        float acc = part[e];
        for (int s = 1; s < S; ++s) acc += part[(int64_t)s * total + e];
        const int64_t i = e % M, j = e / M;
        float *p = C + i + j * ldc;
        *p = beta != 0.f ? fmaf(alpha, acc, beta * *p) : alpha * acc;
    }
}

// ----------------------------------------------------------------- host --
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D map over [terms][rows][kpad] (K innermost), box = BK x box_rows x 1.
// term_stride: elements between terms (0: rows * kpad, a whole packed
// operand; larger when the rows are a range of a bigger packed operand).
bool make_map(CUtensorMap *map, int fmt, const void *ptr, int64_t k, int64_t rows, int64_t kpad,
              int parts, int box_rows, int bk, int row_bytes, int64_t term_stride = 0) {
    auto enc = get_encode();
    if (!enc) return false;
    const bool tf32 = fmt == kFmtTF32;
    const int eb = tf32 ? 4 : 2;
    cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)parts};
    const int64_t ts = term_stride > 0 ? term_stride : rows * kpad;
    cuuint64_t strides[2] = {(cuuint64_t)(kpad * eb), (cuuint64_t)(ts * eb)};
    cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : fmt == kFmtF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(map, dt,
                     3, const_cast<void *>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE,
                     row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int MODE, int RB, int EPI = 0>
cudaError_t launch_mode(const TcArgs &a, cudaStream_t s) {
    using CF = Cfg<MODE, RB>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_sgemm_kernel<MODE, RB, EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    // The tensor maps address rows/K with 32-bit coordinates.
    if (a.m > 2147483647LL || a.n > 2147483647LL || a.k > 2147483647LL)
        return cudaErrorNotSupported;
    alignas(64) CUtensorMap ma, mb;
    if (!make_map(&ma, CF::FMT, a.Ap, a.k, a.m, a.kpad, CF::A_PARTS, BM, CF::BK, RB,
                  a.a_part_stride) ||
        !make_map(&mb, CF::FMT, a.Bp, a.k, a.n, a.kpad, CF::B_PARTS, CF::BN, CF::BK, RB,
                  a.b_part_stride))
        return cudaErrorInvalidValue;
    const int splits = a.part ? (a.splits > 1 ? a.splits : 1) : 1;
    const int64_t units = ((a.m + BM - 1) / BM) * ((a.n + CF::BN - 1) / CF::BN) * splits;
    if (units > 2147483647LL) return cudaErrorNotSupported;   // device raster is 32-bit
    int grid = a.sm_count > 0 ? a.sm_count : 1;
    if (units < grid) grid = (int)units;
    const uint64_t limit_ns = (uint64_t)a.wait_limit * 1000ull;
    if (EPI != 0 && splits > 1) return cudaErrorNotSupported;
    tc_sgemm_kernel<MODE, RB, EPI><<<grid, NUM_THREADS, CF::SMEM_BYTES, s>>>(
        ma, mb, a.m, a.n, a.k, a.alpha, a.beta, a.C, a.ldc, splits > 1 ? a.part : nullptr, splits,
        a.dstate, limit_ns, a.epi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    return launch_splitk_reduce(a.m, a.n, splits, a.part, a.alpha, a.beta, a.C, a.ldc, s);
}

template <int MODE>
cudaError_t launch_promo_mode(const TcArgs &a, cudaStream_t s) {
    using CF = PromoCfg<MODE>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        // The kernel moves registers between its warpgroups (setmaxnreg):
        // launched with fewer than REG_LAUNCH_MIN per thread, the epilogue
        // warpgroups' request could never be met. Refuse rather than launch.
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, tc_promo_kernel<MODE>);
        if (e != cudaSuccess) return e;
        if (fa.numRegs < CF::REG_LAUNCH_MIN || fa.maxThreadsPerBlock < CF::THREADS)
            return cudaErrorNotSupported;
        e = cudaFuncSetAttribute(tc_promo_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    if (a.m > 2147483647LL || a.n > 2147483647LL || a.k > 2147483647LL)
        return cudaErrorNotSupported;
    alignas(64) CUtensorMap ma, mb;
    if (!make_map(&ma, CF::FMT, a.Ap, a.k, a.m, a.kpad, CF::A_PARTS, BM, CF::BK, CF::ROW_BYTES,
                  a.a_part_stride) ||
        !make_map(&mb, CF::FMT, a.Bp, a.k, a.n, a.kpad, CF::B_PARTS, CF::BN, CF::BK, CF::ROW_BYTES,
                  a.b_part_stride))
        return cudaErrorInvalidValue;
    const int splits = a.part ? (a.splits > 1 ? a.splits : 1) : 1;
    const int64_t units = ((a.m + BM - 1) / BM) * ((a.n + CF::BN - 1) / CF::BN) * splits;
    if (units > 2147483647LL) return cudaErrorNotSupported;
    int grid = a.sm_count > 0 ? a.sm_count : 1;
    if (units < grid) grid = (int)units;
    // no promotion asked for (the scaled FP16 split runs only here): one
    // chunk spans the whole K range of a unit
    const int64_t nkb = (a.k + CF::BK - 1) / CF::BK;
    const int chunk_kb = a.promote_kb > 0 ? a.promote_kb : (int)(nkb < 1 ? 1 : nkb);
    if (MODE == 4 && (!a.amax || !a.bmax)) return cudaErrorInvalidValue;
    tc_promo_kernel<MODE><<<grid, CF::THREADS, CF::SMEM_BYTES, s>>>(
        ma, mb, a.m, a.n, a.k, a.alpha, a.beta, a.C, a.ldc, splits > 1 ? a.part : nullptr, splits,
        chunk_kb, a.amax, a.bmax, a.dstate, (uint64_t)a.wait_limit * 1000ull);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    return launch_splitk_reduce(a.m, a.n, splits, a.part, a.alpha, a.beta, a.C, a.ldc, s);
}

template <int MODE, int V>
cudaError_t launch_grouped_mode(const TcProblem *probs, const TcItem *items, int64_t nitems,
                                int sm_count, DeviceState *dstate, int64_t wait_limit,
                                cudaStream_t s) {
    using CF = GroupedCfgV<MODE, V>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_grouped_kernel<MODE, V>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    int grid = sm_count > 0 ? CF::CTAS * sm_count : 1;    // persistent: CTAS per SM
    if (nitems < grid) grid = (int)nitems;
    tc_grouped_kernel<MODE, V><<<grid, NUM_THREADS, CF::SMEM_BYTES, s>>>(
        probs, items, nitems, dstate, (uint64_t)wait_limit * 1000ull);
    return cudaGetLastError();
}

template <int V>
cudaError_t launch_grouped_v(int mode, const TcProblem *probs, const TcItem *items,
                             int64_t nitems, int sm_count, DeviceState *dstate,
                             int64_t wait_limit, cudaStream_t s) {
    switch (mode) {
        case 0: return launch_grouped_mode<0, V>(probs, items, nitems, sm_count, dstate, wait_limit, s);
        case 1: return launch_grouped_mode<1, V>(probs, items, nitems, sm_count, dstate, wait_limit, s);
        case 2: return launch_grouped_mode<2, V>(probs, items, nitems, sm_count, dstate, wait_limit, s);
        case 3: return launch_grouped_mode<3, V>(probs, items, nitems, sm_count, dstate, wait_limit, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_splitk_reduce(int64_t m, int64_t n, int S, const float *part, float alpha,
                                 float beta, float *C, int64_t ldc, cudaStream_t s) {
    const int64_t total = m * n;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    splitk_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, n, S, part, alpha, beta, C, ldc);
    return cudaGetLastError();
}

int tc_tile_n(int mode, bool rb128) { return (mode >= 2 && mode <= 3 && rb128) ? 128 : 256; }

bool tc_make_operand_map(CUtensorMap *map, int mode, bool rb128, const void *packed, int64_t k,
                         int64_t rows, bool a_side) {
    const int rb = rb128 ? 128 : 64;
    const bool tf32 = mode == 0;
    const int bk = rb / (tf32 ? 4 : 2);
    return make_map(map, tf32 ? kFmtTF32 : kFmtBF16, packed, k, rows, split_kpad(mode, k),
                    split_parts(mode),
                    a_side ? BM : tc_tile_n(mode, rb128), bk, rb);
}

// Tile width and row width of grouped configuration v (the same for every
// split mode: the configurations differ in shape, not in terms).
int tc_grouped_tile_n(int v) {
    static_assert(GroupedCfgV<0, 0>::BN == GroupedCfgV<2, 0>::BN &&
                  GroupedCfgV<0, 1>::BN == GroupedCfgV<2, 1>::BN &&
                  GroupedCfgV<0, 2>::BN == GroupedCfgV<2, 2>::BN, "tile width by configuration");
    return v == 1 ? GroupedCfgV<1, 1>::BN : v == 2 ? GroupedCfgV<1, 2>::BN : GroupedCfgV<1, 0>::BN;
}
int tc_grouped_row_bytes(int v) {
    return v == 1 ? GroupedCfgV<1, 1>::ROW_BYTES : v == 2 ? GroupedCfgV<1, 2>::ROW_BYTES
                                                         : GroupedCfgV<1, 0>::ROW_BYTES;
}

bool tc_make_grouped_operand_map(CUtensorMap *map, int mode, int v, const void *packed,
                                 int64_t k, int64_t rows, bool a_side) {
    const int rb = tc_grouped_row_bytes(v);
    const bool tf32 = mode == 0;
    return make_map(map, tf32 ? kFmtTF32 : kFmtBF16, packed, k, rows, split_kpad(mode, k),
                    split_parts(mode), a_side ? BM : tc_grouped_tile_n(v), rb / (tf32 ? 4 : 2),
                    rb);
}

cudaError_t launch_tc_grouped(int mode, int v, const TcProblem *probs, const TcItem *items,
                              int64_t nitems, int sm_count, DeviceState *dstate,
                              int64_t wait_limit, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    switch (v) {
        case 0: return launch_grouped_v<0>(mode, probs, items, nitems, sm_count, dstate, wait_limit, s);
        case 1: return launch_grouped_v<1>(mode, probs, items, nitems, sm_count, dstate, wait_limit, s);
        case 2: return launch_grouped_v<2>(mode, probs, items, nitems, sm_count, dstate, wait_limit, s);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
// The row width forced by GB_SGEMM_TC_ROW_BYTES (64 or 128), read once; 0 if none.
int forced_row_bytes() {
    static const int forced = [] {
        const char *e = getenv("GB_SGEMM_TC_ROW_BYTES");
        const int v = e ? atoi(e) : 0;
        return (v == 64 || v == 128) ? v : 0;
    }();
    return forced;
}
}  // namespace

// Shared-memory row width of a k-block for one GEMM. 64-byte rows (64-byte
// swizzle; 2 terms: four 48 KiB stages; 3 terms: three 72 KiB stages with
// 256-column tiles) measured faster than 128-byte rows (two 96 KiB stages;
// 3 terms: 128-column tiles) for both 2-term splits at every K (8192^2,
// K = 1024: BF16 0.275 against 0.298 ms, TF32 0.478 against 0.543; 4096^2
// and 2048 x 8192 likewise or equal), and for 3 terms wherever the
// 256-column tiling has at least 1024 tiles (8192^2, K = 1024: 0.449 against
// 0.506 ms); with fewer tiles the 3-term modes keep 128-column tiles for a
// fuller last round (4096^2, K = 1024: 0.152 against 0.155 ms). K <= 128
// (one or two k-blocks) keeps 128-byte rows: 8192^2 x 64 TF32 0.074 against
// 0.081 ms, BF16 x 3 terms 0.075 against 0.078. The environment variable
// GB_SGEMM_TC_ROW_BYTES = 64 or 128 forces one of them.
bool tc_rb128(int mode, int64_t m, int64_t n, int64_t k) {
    if (mode == 4) return false;       // the scaled FP16 split runs 64-byte rows only
    if (const int forced = forced_row_bytes()) return forced == 128;
    if (k <= 128) return true;
    if (k > 2048 || mode <= 1) return false;
    return ((m + BM - 1) / BM) * ((n + 255) / 256) < 1024;
}

int tc_promo_kblock(int mode) { return mode == 0 ? PromoCfg<0>::BK : PromoCfg<1>::BK; }

cudaError_t launch_tc_sgemm(const TcArgs &a, cudaStream_t s) {
    if (a.promote_kb > 0 || a.mode == 4) {
        if (a.epi.kind != 0) return cudaErrorNotSupported;
        switch (a.mode) {
            case 0: return launch_promo_mode<0>(a, s);
            case 1: return launch_promo_mode<1>(a, s);
            case 2: return launch_promo_mode<2>(a, s);
            case 3: return launch_promo_mode<3>(a, s);
            case 4: return launch_promo_mode<4>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    // the environment's width, else the tuned one, else the rule
    const bool rb128 = (forced_row_bytes() || a.row_bytes == 0) ? tc_rb128(a.mode, a.m, a.n, a.k)
                                                                : a.row_bytes == 128;
    if (a.epi.kind != 0) {
        // fused elementwise operations: BF16 x 2 terms and x 3 terms (6 products)
        const int key = a.mode * 10 + a.epi.kind;
        switch (key) {
            case 11: return rb128 ? launch_mode<1, 128, 1>(a, s) : launch_mode<1, 64, 1>(a, s);
            case 12: return rb128 ? launch_mode<1, 128, 2>(a, s) : launch_mode<1, 64, 2>(a, s);
            case 21: return rb128 ? launch_mode<2, 128, 1>(a, s) : launch_mode<2, 64, 1>(a, s);
            case 22: return rb128 ? launch_mode<2, 128, 2>(a, s) : launch_mode<2, 64, 2>(a, s);
            default: return cudaErrorNotSupported;
        }
    }
    switch (a.mode) {
        case 0: return rb128 ? launch_mode<0, 128>(a, s) : launch_mode<0, 64>(a, s);
        case 1: return rb128 ? launch_mode<1, 128>(a, s) : launch_mode<1, 64>(a, s);
        case 2: return rb128 ? launch_mode<2, 128>(a, s) : launch_mode<2, 64>(a, s);
        case 3: return rb128 ? launch_mode<3, 128>(a, s) : launch_mode<3, 64>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
