// FP32 operand tiles read by TMA straight from a caller's column-major
// matrix, and their conversion in shared memory into the BF16 terms that
// tcgen05.mma reads. Shared by the kernels that split inside the kernel
// instead of in a separate pack pass (the paper's re-buffering of B', Sec. 3,
// moved between L2 and the tensor cores).
#pragma once

#include <cudaTypedefs.h>

#include "split_common.cuh"
#include "tc_ptx.cuh"

namespace gb {
namespace fx {

constexpr int FBK = 32;        // k per stage: 32 FP32 = 128 B, 32 BF16 = 64 B

// Reads 8 consecutive k (8*chunk .. 8*chunk+7) of one row of an FP32 tile.
// kc: tile is [rows][32] with 128-byte rows, 16-byte chunks XOR-swizzled by
// row % 8 (TMA 128-byte swizzle); else [32][ROWS] (k-major, no swizzle).
template <int ROWS>
__device__ __forceinline__ void read8(const float *tile, bool kc, int row, int chunk, float v[8]) {
    if (kc) {
        const float *rp = tile + row * 32;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int phys = (2 * chunk + h) ^ (row & 7);
            const float4 q = *reinterpret_cast<const float4 *>(rp + phys * 4);
            v[4 * h + 0] = q.x; v[4 * h + 1] = q.y; v[4 * h + 2] = q.z; v[4 * h + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = tile[(8 * chunk + e) * ROWS + row];
    }
}

// Splits the 8 values and stores each term as one 16-byte chunk of row `row`
// in the K-major operand tile of that term: 64-byte rows, chunk index XOR
// (row / 2) % 4 (the 64-byte swizzle tcgen05 descriptors expect). The split
// is the pack pass's (split2_bf16), so the terms are bit-identical to it.
// FAST: the caller has checked that all 8 values take the fast path
// (max_abs_bits below kBf16FastLimit), so no per-pair branch.
template <int PARTS, bool FAST = false>
__device__ __forceinline__ void write8(uint8_t *op0, int op_bytes, int row, int chunk,
                                       const float v[8]) {
    uint32_t w[PARTS][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        uint32_t pr[PARTS];
        if (FAST) split2_bf16_fast<PARTS>(v[e], v[e + 1], pr);
        else      split2_bf16<PARTS>(v[e], v[e + 1], pr);
#pragma unroll
        for (int p = 0; p < PARTS; ++p) w[p][e / 2] = pr[p];
    }
    const int off = row * 64 + ((chunk ^ ((row >> 1) & 3)) * 16);
#pragma unroll
    for (int p = 0; p < PARTS; ++p)
        *reinterpret_cast<uint4 *>(op0 + p * op_bytes + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2-D map over a caller's column-major FP32 matrix (rows_stored x
// cols_stored, ld). kc: the tile is (32 k) x (box_rows rows) read along K
// (x = k, y = row, 128-byte swizzle); else (box_rows rows) x (32 k) read
// along the rows (x = row, y = k, no swizzle).
inline bool make_f32_map(CUtensorMap *map, const float *ptr, int64_t rows_stored,
                         int64_t cols_stored, int64_t ld, bool kc, int box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows_stored, (cuuint64_t)cols_stored};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {kc ? (cuuint32_t)FBK : (cuuint32_t)box_rows,
                         kc ? (cuuint32_t)box_rows : (cuuint32_t)FBK};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     kc ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// TMA can read an FP32 operand in place: 16-byte aligned base, leading
// dimension a multiple of 4 elements (16-byte strides).
inline bool f32_tma_ok(const float *X, int64_t ldx) {
    return !(reinterpret_cast<uintptr_t>(X) & 15) && ldx % 4 == 0 && ldx < ((int64_t)1 << 37);
}

}  // namespace fx
}  // namespace gb
