// Measurement aid: the FP32 FMA roofline of the device, measured rather than
// taken from the data sheet (SMs x 128 FMA lanes x 2 flops x clock under the
// clocks the chip actually holds while busy).
#include <stdint.h>

#include "internal.h"

namespace gb {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (covers the FMA latency)

__global__ void __launch_bounds__(256)
ffma_kernel(int64_t iterations, float b, float c, float *__restrict__ sink) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int64_t it = 0; it < iterations; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains live, never taken in practice
}

}  // namespace
}  // namespace gb

extern "C" GB_API int gb_measure_ffma(gb_handle_t h, int64_t iterations, float *sink,
                                      int64_t *fmas, void *stream) {
    using namespace gb;
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    if (iterations < 1 || !sink || !fmas) return GB_ERR_ARG;
    const int blocks = h->sm_count * 8;
    ffma_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iterations, 0.9999f, 1e-4f,
                                                                       sink);
    *fmas = (int64_t)blocks * 256 * iterations * 16 * kChains;
    return cudaGetLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}
