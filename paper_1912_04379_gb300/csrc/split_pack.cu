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
#include "split_common.cuh"

namespace gb {
namespace {

// Splits four consecutive k of one row and stores each term as one vector:
// 4 TF32 words (16 bytes) or 4 BF16 / FP16 values (8 bytes). idx is a
// multiple of 4 and rows start on 16-byte boundaries, so the stores are
// aligned. Modes 4 and 5 are the scaled FP16 split of op(A) and of op(B)^T:
// each value is first scaled by 2^e, the row's exponent, then split as
// x = h + l 2^-11; op(A) stores (2^11 h, h, l), op(B)^T stores (h, l).
template <int MODE>
__device__ __forceinline__ void split_store4(const float v[4], void *out, int64_t ps, int64_t idx,
                                             int e) {
    if (MODE == 4 || MODE == 5) {
        __half h[4], l[4], h11[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            split_fp16(scale_pow2(v[i], -e), h[i], l[i]);
            h11[i] = __float2half_rn(__half2float(h[i]) * 2048.f);   // exact: |h| <= 2^4
        }
        __half *o = static_cast<__half *>(out) + idx;
        auto put = [&](__half *dst, const __half t[4]) {
            __half2 a = __halves2half2(t[0], t[1]), b = __halves2half2(t[2], t[3]);
            *reinterpret_cast<uint2 *>(dst) =
                make_uint2(*reinterpret_cast<const uint32_t *>(&a), *reinterpret_cast<const uint32_t *>(&b));
        };
        if (MODE == 4) {
            put(o, h11);
            put(o + ps, h);
            put(o + 2 * ps, l);
        } else {
            put(o, h);
            put(o + ps, l);
        }
    } else if (MODE == 0) {
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = tf32_rne(v[i]);
            l[i] = isfinite(v[i]) ? tf32_rne(v[i] - h[i]) : 0.f;
        }
        float *o = static_cast<float *>(out) + idx;
        *reinterpret_cast<float4 *>(o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(o + ps) = make_float4(l[0], l[1], l[2], l[3]);
    } else {
        constexpr int P = MODE == 2 ? 3 : 2;
        uint32_t lo[P], hi[P];
        split2_bf16<P>(v[0], v[1], lo);
        split2_bf16<P>(v[2], v[3], hi);
        __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(out) + idx;
#pragma unroll
        for (int p = 0; p < P; ++p) *reinterpret_cast<uint2 *>(o + p * ps) = make_uint2(lo[p], hi[p]);
    }
}

// Source contiguous along K (element (r,p) at X[p + r*ld]): no transpose.
// Each thread splits 4 consecutive k of one row: 16-byte loads when the
// source is 16-byte aligned, vector stores of every term. blockIdx.y walks
// rows, blockIdx.x the k-quads of a row.
// The row's scaling exponent of the FP16 split (0 for the other modes).
template <int MODE>
__device__ __forceinline__ int row_exp(const uint32_t *mx, int64_t r) {
    if (MODE == 4) return fp16_row_exp(mx[r], kFp16TopA);
    if (MODE == 5) return fp16_row_exp(mx[r >> kFp16ColBlockLog2], kFp16TopB);
    return 0;
}

template <int MODE, bool VEC>
__global__ void __launch_bounds__(256)
split_pack_kc_kernel(int64_t rows, int64_t K, const float *__restrict__ X, int64_t ld,
                     void *__restrict__ out, int64_t kpad, int64_t ps,
                     const uint32_t *__restrict__ mx) {
    // a kernel launched after this one as its programmatic dependent (the
    // skinny kernel) may start now; it waits for this grid before it reads
    // what this grid writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t p = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 4;
    if (p >= kpad) return;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const int e = row_exp<MODE>(mx, r);
        const float *src = X + r * ld + p;
        float v[4];
        if (VEC && p + 3 < K) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(src));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = p + i < K ? __ldg(src + i) : 0.f;
        }
        split_store4<MODE>(v, out, ps, r * kpad + p, e);
    }
}

// One 64 x 64 (rows x k) tile through shared memory. Loads are coalesced
// along whichever dimension the source is contiguous in (16 threads cover 64
// consecutive floats, 16-byte loads when vec); stores are coalesced along k
// (16 threads cover 64 consecutive k of one row, 4 per thread, one vector per
// term). kc: element (r,p) at X[p + r*ld]; otherwise at X[r + p*ld].
template <int MODE>
__device__ __forceinline__ void pack_tile64(const float *__restrict__ X, int64_t ld, bool kc,
                                            bool vec, int64_t rows, int64_t K,
                                            void *__restrict__ out, int64_t kpad, int64_t ps,
                                            int64_t r0, int64_t p0, float (*T)[65],
                                            const uint32_t *__restrict__ mx = nullptr) {
    const int t = threadIdx.x;
    const int l4 = (t & 15) * 4, l16 = t >> 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float v[4];
        if (!kc) {
            const int pl = l16 + 16 * e;                 // T[pl][l4 .. l4+3]
            const int64_t pp = p0 + pl, rr = r0 + l4;
            if (vec && pp < K && rr + 3 < rows) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(X + rr + pp * ld));
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    v[i] = (pp < K && rr + i < rows) ? __ldg(X + rr + i + pp * ld) : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) T[pl][l4 + i] = v[i];
        } else {
            const int rl = l16 + 16 * e;                 // T[l4 .. l4+3][rl]
            const int64_t rr = r0 + rl, pp = p0 + l4;
            if (vec && rr < rows && pp + 3 < K) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(X + pp + rr * ld));
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    v[i] = (rr < rows && pp + i < K) ? __ldg(X + pp + i + rr * ld) : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) T[l4 + i][rl] = v[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int rl = l16 + 16 * e;
        const int64_t rr = r0 + rl, pp = p0 + l4;
        if (rr < rows && pp < kpad) {
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = T[l4 + i][rl];
            split_store4<MODE>(v, out, ps, rr * kpad + pp, row_exp<MODE>(mx, rr));
        }
    }
    __syncthreads();                                     // T is reused by the next tile
}

// Source contiguous along the rows (element (r,p) at X[r + p*ld]): one
// 64 x 64 tile per CTA, transposed through shared memory.
template <int MODE, bool VEC>
__global__ void __launch_bounds__(256)
split_pack_rc_kernel(int64_t rows, int64_t K, const float *__restrict__ X, int64_t ld,
                     void *__restrict__ out, int64_t kpad, int64_t ps,
                     const uint32_t *__restrict__ mx) {
    __shared__ float T[64][65];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // as above
    pack_tile64<MODE>(X, ld, false, VEC, rows, K, out, kpad, ps, (int64_t)blockIdx.y * 64,
                      (int64_t)blockIdx.x * 64, T, mx);
}

// Largest finite |x| of each row of a rows x K operand, as FP32 bits
// (non-negative floats order like their bit patterns), combined by atomicMax
// into mx[r >> shift] (which starts at 0) over slices of K; shift > 0 takes
// the maximum over blocks of 2^shift rows.
// Rows-contiguous source (element (r,p) at X[r + p*ld]): one thread per row,
// coalesced along the rows.
__global__ void __launch_bounds__(256)
rowmax_rc_kernel(int64_t rows, int64_t K, const float *__restrict__ X, int64_t ld,
                 uint32_t *__restrict__ mx, int64_t kslice, int shift) {
    const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (r >= rows) return;
    const int64_t p0 = (int64_t)blockIdx.y * kslice;
    const int64_t p1 = p0 + kslice < K ? p0 + kslice : K;
    uint32_t m = 0;
#pragma unroll 8
    for (int64_t p = p0; p < p1; ++p) {
        const uint32_t u = __float_as_uint(__ldg(X + r + p * ld)) & 0x7fffffffu;
        if (u < 0x7f800000u && u > m) m = u;
    }
    if (m) atomicMax(mx + (r >> shift), m);
}

// K-contiguous source (element (r,p) at X[p + r*ld]): one warp per row.
__global__ void __launch_bounds__(256)
rowmax_kc_kernel(int64_t rows, int64_t K, const float *__restrict__ X, int64_t ld,
                 uint32_t *__restrict__ mx, int64_t kslice, int shift) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    const int64_t p0 = (int64_t)blockIdx.y * kslice;
    const int64_t p1 = p0 + kslice < K ? p0 + kslice : K;
    uint32_t m = 0;
#pragma unroll 4
    for (int64_t p = p0 + lane; p < p1; p += 32) {
        const uint32_t u = __float_as_uint(__ldg(X + p + r * ld)) & 0x7fffffffu;
        if (u < 0x7f800000u && u > m) m = u;
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0 && m) atomicMax(mx + (r >> shift), m);
}

// A K-contiguous 64 x 64 tile straight from registers: each thread loads four
// consecutive k of a row (as pack_tile64 would) and splits and stores exactly
// those, so the shared-memory round trip and its barriers are not needed.
template <int MODE>
__device__ __forceinline__ void pack_tile64_kc_direct(const PackItem &it) {
    const int t = threadIdx.x;
    const int l4 = (t & 15) * 4, l16 = t >> 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t rr = it.r0 + l16 + 16 * e, pp = it.p0 + l4;
        if (rr >= it.rows || pp >= it.kpad) continue;
        const float *src = it.X + pp + rr * it.ld;
        float v[4];
        if (it.vec && pp + 3 < it.k) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(src));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = pp + i < it.k ? __ldg(src + i) : 0.f;
        }
        split_store4<MODE>(v, it.out, it.ps, rr * it.kpad + pp, 0);
    }
}

// Grouped pass: each CTA walks a list of 64 x 64 tiles of many operands,
// each tile with its own split mode and source order (both branches are
// uniform over the CTA; only the rows-contiguous tiles use shared memory).
__global__ void __launch_bounds__(256)
split_pack_grouped_kernel(const PackItem *__restrict__ items, int64_t nitems) {
    __shared__ float T[64][65];
    for (int64_t i = blockIdx.x; i < nitems; i += gridDim.x) {
        const PackItem it = items[i];
        if (it.kc) {
            if (it.mode == 0)      pack_tile64_kc_direct<0>(it);
            else if (it.mode == 1) pack_tile64_kc_direct<1>(it);
            else                   pack_tile64_kc_direct<2>(it);
            continue;
        }
        if (it.mode == 0)
            pack_tile64<0>(it.X, it.ld, it.kc != 0, it.vec != 0, it.rows, it.k, it.out, it.kpad,
                           it.ps, it.r0, it.p0, T);
        else if (it.mode == 1)
            pack_tile64<1>(it.X, it.ld, it.kc != 0, it.vec != 0, it.rows, it.k, it.out, it.kpad,
                           it.ps, it.r0, it.p0, T);
        else
            pack_tile64<2>(it.X, it.ld, it.kc != 0, it.vec != 0, it.rows, it.k, it.out, it.kpad,
                           it.ps, it.r0, it.p0, T);
    }
}

template <int MODE>
cudaError_t launch_mode(bool kc, int64_t rows, int64_t k, const float *X, int64_t ld, void *out,
                        int64_t kpad, int64_t ps, const uint32_t *mx, cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0 && ld % 4 == 0;
    if (kc) {
        const int64_t gx = (kpad / 4 + 255) / 256;
        const int64_t gy = rows < 65535 ? rows : 65535;
        if (gx > 2147483647LL) return cudaErrorInvalidConfiguration;
        dim3 grid((unsigned)gx, (unsigned)gy);
        if (vec) split_pack_kc_kernel<MODE, true><<<grid, 256, 0, s>>>(rows, k, X, ld, out, kpad, ps, mx);
        else     split_pack_kc_kernel<MODE, false><<<grid, 256, 0, s>>>(rows, k, X, ld, out, kpad, ps, mx);
    } else {
        const int64_t gx = (kpad + 63) / 64, gy = (rows + 63) / 64;
        if (gx > 2147483647LL || gy > 65535LL) return cudaErrorInvalidConfiguration;
        dim3 grid((unsigned)gx, (unsigned)gy);
        if (vec) split_pack_rc_kernel<MODE, true><<<grid, 256, 0, s>>>(rows, k, X, ld, out, kpad, ps, mx);
        else     split_pack_rc_kernel<MODE, false><<<grid, 256, 0, s>>>(rows, k, X, ld, out, kpad, ps, mx);
    }
    return cudaGetLastError();
}

// mx[r >> shift] = largest finite |x| of the rows r of a block of 2^shift
// (FP32 bits; 0 if none). About two waves of 256-thread CTAs over (row
// blocks) x (K slices).
cudaError_t launch_row_max(bool kc, int64_t rows, int64_t k, const float *X, int64_t ld,
                           uint32_t *mx, int shift, cudaStream_t s) {
    const int64_t nmx = ((rows - 1) >> shift) + 1;
    cudaError_t e = cudaMemsetAsync(mx, 0, (size_t)nmx * sizeof(uint32_t), s);
    if (e != cudaSuccess || k <= 0) return e;
    const int64_t per_block = kc ? 8 : 256;                  // rows per CTA
    const int64_t gx = (rows + per_block - 1) / per_block;
    if (gx > 2147483647LL) return cudaErrorInvalidConfiguration;
    int64_t gy = (2432 + gx - 1) / gx;
    if (gy > 65535) gy = 65535;
    int64_t kslice = (k + gy - 1) / gy;
    if (kslice < 64) kslice = 64;
    gy = (k + kslice - 1) / kslice;
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (kc) rowmax_kc_kernel<<<grid, 256, 0, s>>>(rows, k, X, ld, mx, kslice, shift);
    else    rowmax_rc_kernel<<<grid, 256, 0, s>>>(rows, k, X, ld, mx, kslice, shift);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split_pack_grouped(const PackItem *items, int64_t nitems, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    const int grid = (int)(nitems < 65536 ? nitems : 65536);
    split_pack_grouped_kernel<<<grid, 256, 0, s>>>(items, nitems);
    return cudaGetLastError();
}

int split_parts(int mode) { return mode >= 2 ? 3 : 2; }
int split_parts_side(int mode, bool a_side) { return mode == 4 ? (a_side ? 3 : 2) : split_parts(mode); }
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
        case 0: return launch_mode<0>(kcontig, rows, k, X, ld, out, kpad, ps, nullptr, s);
        case 1: return launch_mode<1>(kcontig, rows, k, X, ld, out, kpad, ps, nullptr, s);
        case 2:
        case 3: return launch_mode<2>(kcontig, rows, k, X, ld, out, kpad, ps, nullptr, s);   // same terms
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_split_pack_fp16(bool a_side, bool kcontig, int64_t rows, int64_t k,
                                   const float *X, int64_t ld, void *out, int64_t kpad,
                                   int64_t ps, uint32_t *mx, cudaStream_t s) {
    if (rows <= 0 || kpad <= 0) return cudaSuccess;
    // op(A): one maximum per row; op(B)^T: one per block of kFp16ColBlock rows
    cudaError_t e = launch_row_max(kcontig, rows, k, X, ld, mx, a_side ? 0 : kFp16ColBlockLog2, s);
    if (e != cudaSuccess) return e;
    return a_side ? launch_mode<4>(kcontig, rows, k, X, ld, out, kpad, ps, mx, s)
                  : launch_mode<5>(kcontig, rows, k, X, ld, out, kpad, ps, mx, s);
}

}  // namespace gb
