// Split/pack pass of the split-precision SGEMM.
//
// Each FP32 element a of op(A) (and of op(B)^T) is written as a sum of
// lower-precision terms that the tensor cores can multiply:
//   TF32 x 2 : a ~ h + l,        h = rn_tf32(a), l = rn_tf32(a - h)
//   BF16 x 2 : a ~ h + l,        h = rn_bf16(a), l = rn_bf16(a - h)
//   BF16 x 3 : a = h + m + l,    h = rn_bf16(a), m = rn_bf16(a - h), l = rn_bf16(a - h - m)
// Each difference is exact in FP32 (the rounded term is within a factor of
// two of what it rounds, so the subtraction is exact by Sterbenz's lemma),
// so BF16 x 3 reproduces every FP32 value exactly (8 + 8 + 8 >= 24 bits).
// Rounding is to nearest, ties to even. A non-finite a gives (a, 0[, 0]);
// a finite a whose leading term would round to infinity keeps its leading
// term truncated toward zero instead, so the split stays finite and exact.
//
// The pass also re-lays the data out, as the paper re-buffers B' into a
// contiguous block (Sec. 3): whatever the transpose flag and leading
// dimension, term t of row r, k-index p lands at out[t*part_stride + r*kpad + p]
// (K contiguous, rows padded to kpad elements so every row starts on a
// 16-byte boundary). That is the K-major layout the TMA loads of the
// tensor-core kernel read, independent of the caller's storage order.
#include <cuda_bf16.h>

#include "internal.h"

namespace gb {
namespace {

constexpr int TILE = 32;

__device__ __forceinline__ float tf32_rne(float a) {
    // Round to 10 explicit mantissa bits, nearest-even, by integer arithmetic
    // on the encoding: add half an ulp of the target precision (minus one,
    // plus the target's lowest kept bit), then clear the 13 dropped bits.
    uint32_t u = __float_as_uint(a);
    if ((u & 0x7f800000u) == 0x7f800000u) return a;
    const uint32_t r = u + 0x0fffu + ((u >> 13) & 1u);
    if ((r & 0x7f800000u) == 0x7f800000u) return __uint_as_float(u & 0xffffe000u);  // truncate
    return __uint_as_float(r & 0xffffe000u);
}

__device__ __forceinline__ __nv_bfloat16 bf16_rne(float a) {
    if (!isfinite(a)) return __float2bfloat16_rn(a);
    __nv_bfloat16 h = __float2bfloat16_rn(a);
    if (isinf(__bfloat162float(h)))                    // overflowed: truncate instead
        h = __float2bfloat16_rz(a);
    return h;
}

template <int MODE>
__device__ __forceinline__ void split_store(float a, void *out, int64_t part_stride, int64_t idx) {
    if (MODE == 0) {
        float *o = static_cast<float *>(out);
        float h = tf32_rne(a);
        float l = isfinite(a) ? tf32_rne(a - h) : 0.f;
        o[idx] = h;
        o[idx + part_stride] = l;
    } else {
        __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(out);
        const __nv_bfloat16 h = bf16_rne(a);
        const float hf = __bfloat162float(h);
        const bool fin = isfinite(a);
        const float r1 = fin ? a - hf : 0.f;
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        o[idx] = h;
        o[idx + part_stride] = m;
        if (MODE == 2) {
            const float r2 = fin ? r1 - __bfloat162float(m) : 0.f;
            o[idx + 2 * part_stride] = __float2bfloat16_rn(r2);
        }
    }
}

// One 32 x 32 (rows x k) tile per CTA of 256 threads. Reads are coalesced
// along whichever dimension is contiguous in the source; writes are
// coalesced along k.
template <int MODE, bool KC>
__global__ void __launch_bounds__(256)
split_pack_kernel(int64_t rows, int64_t K, const float *__restrict__ X, int64_t ld,
                  void *__restrict__ out, int64_t kpad, int64_t part_stride) {
    __shared__ float T[TILE][TILE + 1];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * TILE;
    const int64_t r0 = (int64_t)blockIdx.y * TILE;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        int r, p;
        if (KC) { p = lx; r = ly + 8 * e; }
        else    { r = lx; p = ly + 8 * e; }
        const int64_t rr = r0 + r, pp = p0 + p;
        float v = 0.f;
        if (rr < rows && pp < K) v = KC ? __ldg(X + pp + rr * ld) : __ldg(X + rr + pp * ld);
        T[r][p] = v;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int r = ly + 8 * e, p = lx;
        const int64_t rr = r0 + r, pp = p0 + p;
        if (rr < rows && pp < kpad) split_store<MODE>(T[r][p], out, part_stride, rr * kpad + pp);
    }
}

template <int MODE>
cudaError_t launch_mode(bool kc, int64_t rows, int64_t k, const float *X, int64_t ld, void *out,
                        int64_t kpad, int64_t ps, cudaStream_t s) {
    const int64_t gx = (kpad + TILE - 1) / TILE, gy = (rows + TILE - 1) / TILE;
    if (gx > 2147483647LL || gy > 65535LL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (kc) split_pack_kernel<MODE, true><<<grid, 256, 0, s>>>(rows, k, X, ld, out, kpad, ps);
    else    split_pack_kernel<MODE, false><<<grid, 256, 0, s>>>(rows, k, X, ld, out, kpad, ps);
    return cudaGetLastError();
}

}  // namespace

int split_parts(int mode) { return mode == 2 ? 3 : 2; }
int split_elem_bytes(int mode) { return mode == 0 ? 4 : 2; }
int64_t split_kpad(int mode, int64_t k) {
    // rows start on 16-byte boundaries: 4 TF32 words or 8 BF16 values
    const int64_t q = mode == 0 ? 4 : 8;
    const int64_t kk = k < 1 ? 1 : k;
    return (kk + q - 1) / q * q;
}

cudaError_t launch_split_pack(int mode, bool kcontig, int64_t rows, int64_t k, const float *X,
                              int64_t ld, void *out, int64_t kpad, int64_t ps, cudaStream_t s) {
    if (rows <= 0 || kpad <= 0) return cudaSuccess;
    switch (mode) {
        case 0: return launch_mode<0>(kcontig, rows, k, X, ld, out, kpad, ps, s);
        case 1: return launch_mode<1>(kcontig, rows, k, X, ld, out, kpad, ps, s);
        case 2: return launch_mode<2>(kcontig, rows, k, X, ld, out, kpad, ps, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
