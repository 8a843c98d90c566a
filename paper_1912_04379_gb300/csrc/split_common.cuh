// The FP32 -> (BF16 | TF32) term split used by every split-precision path
// (the separate pack pass and the split fused into the tensor-core kernel),
// so that both produce bit-identical terms. Definitions: see split_pack.cu.
#pragma once

#include <cuda_bf16.h>
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
template <int PARTS>
__device__ __forceinline__ void split2_bf16(float a0, float a1, uint32_t w[PARTS]) {
    const uint32_t u0 = __float_as_uint(a0) & 0x7fffffffu, u1 = __float_as_uint(a1) & 0x7fffffffu;
    if ((u0 > u1 ? u0 : u1) >= 0x7f7f8000u) {
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

}  // namespace gb
