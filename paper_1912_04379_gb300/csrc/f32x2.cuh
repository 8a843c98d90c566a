// Paired FP32 arithmetic (sm_100 family): one instruction applies the same
// operation to two FP32 values held as one 64-bit register pair. Each half
// rounds exactly as the scalar instruction does (fma.rn.f32x2 is fmaf twice),
// so a kernel that pairs its FMAs returns the scalar form's bits.
#pragma once

namespace gb {

// d.lo += a.lo * b.lo, d.hi += a.hi * b.hi, each rounded to nearest even
__device__ __forceinline__ void ffma2(unsigned long long &d, unsigned long long a,
                                      unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
    return v;
}

}  // namespace gb
