// The FP32 -> (BF16 | TF32) term split used by every split-precision path
// (the separate pack pass and the split fused into the tensor-core kernel),
// so that both produce bit-identical terms. Definitions: see split_pack.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gb {

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

// a = t[0] + t[1] (+ t[2]) in BF16, each term the round-to-nearest-even of
// what the previous terms leave (exact differences by Sterbenz's lemma); a
// non-finite a gives (a, 0[, 0]).
template <int PARTS>
__device__ __forceinline__ void split_bf16(float a, __nv_bfloat16 t[PARTS]) {
    const bool fin = isfinite(a);
    t[0] = bf16_rne(a);
    const float r1 = fin ? a - __bfloat162float(t[0]) : 0.f;
    t[1] = __float2bfloat16_rn(r1);
    if (PARTS == 3) {
        const float r2 = fin ? r1 - __bfloat162float(t[1]) : 0.f;
        t[PARTS - 1] = __float2bfloat16_rn(r2);
    }
}

// Two elements at once, each term returned as a packed pair (element a0 in
// the low half). Fast path: one paired round-to-nearest conversion per term;
// inputs that are non-finite or could round to infinity in BF16
// (|a| >= 0x7f7f8000 as bits) take split_bf16, so the result is always
// bit-identical to split_bf16 on each element.
// The fast path alone, for callers that have checked that neither input is
// non-finite or near overflow (bf16_fast_ok over all their inputs at once:
// one branch for many pairs lets the pairs' conversions interleave).
template <int PARTS>
__device__ __forceinline__ void split2_bf16_fast(float a0, float a1, uint32_t w[PARTS]) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
    const float r0 = a0 - __low2float(h), r1 = a1 - __high2float(h);
    const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    w[0] = *reinterpret_cast<const uint32_t *>(&h);
    w[1] = *reinterpret_cast<const uint32_t *>(&m);
    if (PARTS == 3) {
        const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m));
        w[PARTS - 1] = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Largest |x| as bits over n values; the fast path applies when it is below
// 0x7f7f8000 (finite and not rounding to infinity in BF16).
template <int N>
__device__ __forceinline__ uint32_t max_abs_bits(const float (&v)[N]) {
    uint32_t m = 0;
#pragma unroll
    for (int e = 0; e < N; ++e) {
        const uint32_t u = __float_as_uint(v[e]) & 0x7fffffffu;
        m = u > m ? u : m;
    }
    return m;
}
constexpr uint32_t kBf16FastLimit = 0x7f7f8000u;

template <int PARTS>
__device__ __forceinline__ void split2_bf16(float a0, float a1, uint32_t w[PARTS]) {
    const uint32_t u0 = __float_as_uint(a0) & 0x7fffffffu, u1 = __float_as_uint(a1) & 0x7fffffffu;
    if ((u0 > u1 ? u0 : u1) >= kBf16FastLimit) {
        __nv_bfloat16 t0[PARTS], t1[PARTS];
        split_bf16<PARTS>(a0, t0);
        split_bf16<PARTS>(a1, t1);
#pragma unroll
        for (int p = 0; p < PARTS; ++p)
            w[p] = (uint32_t)__bfloat16_as_ushort(t0[p]) | ((uint32_t)__bfloat16_as_ushort(t1[p]) << 16);
        return;
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
    const float r0 = a0 - __low2float(h), r1 = a1 - __high2float(h);
    const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    w[0] = *reinterpret_cast<const uint32_t *>(&h);
    w[1] = *reinterpret_cast<const uint32_t *>(&m);
    if (PARTS == 3) {
        const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m));
        w[PARTS - 1] = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// ---------------------------------------------- scaled FP16 split (FP16X3) --
// Each row of op(A), and each block of kFp16ColBlock consecutive columns of
// op(B), is scaled by a power of two 2^e chosen from its largest finite
// magnitude m (kept as FP32 bits, 0 when there is no nonzero finite entry):
// A rows to [2^3, 2^4), B column blocks to [2^14, 2^15), so that every FP16
// term below is finite. e = top - floor(log2 m), with floor(log2 m) read off
// the FP32 encoding (subnormal m included). A column block is the tensor-core
// tile's width, so the epilogue undoes a tile's scaling with one factor per
// row.
constexpr int kFp16TopA = 3, kFp16TopB = 14;
constexpr int kFp16ColBlockLog2 = 8;
constexpr int kFp16ColBlock = 1 << kFp16ColBlockLog2;
// The A side's leading term carries the factor 2^11 of the B side's low term.
constexpr int kFp16LoShift = 11;

__device__ __forceinline__ int fp16_row_exp(uint32_t maxbits, int top) {
    if (maxbits == 0) return 0;
    const uint32_t ef = (maxbits >> 23) & 0xffu;
    const int lg = ef ? (int)ef - 127 : (31 - __clz((int)(maxbits & 0x7fffffu))) - 149;
    return top - lg;
}

// Whether v * 2^-E is exact by moving v's exponent field alone: v normal
// and the result normal.
__device__ __forceinline__ bool pow2_scale_in_range(float v, int E) {
    const int ex = (int)((__float_as_uint(v) >> 23) & 0xffu);
    const int ne = ex - E;
    return ex != 0 && ex != 255 && ne >= 1 && ne <= 254;
}

static __device__ __noinline__ float ldexp_out_of_line(float v, int n) { return ldexpf(v, n); }

// v * 2^-E. For a normal v whose result stays normal this only moves the
// exponent field (exact); zeros, subnormals, infinities, NaNs and results
// leaving the normal range go through ldexpf (out of line: rare).
__device__ __forceinline__ float scale_pow2(float v, int E) {
    if (pow2_scale_in_range(v, E)) {
        const uint32_t u = __float_as_uint(v);
        const int ne = (int)((u >> 23) & 0xffu) - E;
        return __uint_as_float((u & 0x807fffffu) | ((uint32_t)ne << 23));
    }
    return ldexp_out_of_line(v, -E);
}

// x (already scaled) = h + l * 2^-11 with h = rn_fp16(x) and l = rn_fp16((x - h) * 2^11);
// x - h is exact (h is within a factor of two of x, or both are below the
// FP16 normal range where h is a multiple of 2^-24 and x's own grid is finer).
// A non-finite x gives (x, 0).
__device__ __forceinline__ void split_fp16(float x, __half &h, __half &l) {
    h = __float2half_rn(x);
    l = isfinite(x) ? __float2half_rn((x - __half2float(h)) * 2048.f) : __float2half_rn(0.f);
}

}  // namespace gb
