// Error report of an FP32 GEMM result against an FP64 reference.
//
// ratio_ij = |C_ij - C64_ij| / (2 * max(K,1) * 2^-24 * D_ij), where D is the
// bound denominator |alpha||op(A)||op(B)| + |beta||C|. This is the only FP64
// arithmetic the library runs on the GPU.
//
// Pass 1 (err_ratio_kernel) computes every ratio, stores its FP64 bit
// pattern as a 64-bit key (non-negative doubles and +inf sort like their
// encodings) and writes per-block partial results (max, sums, fail count).
// A one-block kernel folds the partials in a fixed order, so the sums do not
// depend on scheduling. The lower median is then found exactly by radix
// selection: eight passes, each histogramming one byte of the keys that
// match the bytes chosen so far, then a one-thread kernel picks the byte
// that holds the target rank.
#include <math.h>
#include <string.h>

#include "internal.h"

namespace gb {
namespace {

constexpr int RT = 256;     // threads per block
struct Partial {
    double max_ratio, sum_sq_diff, sum_sq_ref;
    unsigned long long n_fail;
};
struct SelectState {
    unsigned long long prefix, mask, rank;
};

__device__ __forceinline__ double ratio_of(float c32, double r, double d, double kfac) {
    const double c = (double)c32;
    const bool fin = isfinite(c) && isfinite(r);
    if (!fin) {
        const bool same = (isnan(c) && isnan(r)) || (c == r);
        return same ? 0.0 : INFINITY;
    }
    const double diff = fabs(c - r);
    if (diff == 0.0) return 0.0;
    const double b = kfac * d;
    return b > 0.0 ? diff / b : INFINITY;
}

__global__ void __launch_bounds__(RT)
err_ratio_kernel(int64_t M, int64_t N, double kfac, const float *__restrict__ C, int64_t ldc,
                 const double *__restrict__ R, int64_t ldr, const double *__restrict__ D,
                 int64_t ldd, unsigned long long *__restrict__ keys, Partial *__restrict__ part) {
    __shared__ Partial sp[RT];
    Partial p{0.0, 0.0, 0.0, 0ull};
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * RT + threadIdx.x; e < total; e += (int64_t)gridDim.x * RT) {
        const int64_t i = e % M, j = e / M;
        const float c = C[i + j * ldc];
        const double r = R[i + j * ldr];
        const double d = D[i + j * ldd];
        const double q = ratio_of(c, r, d, kfac);
        keys[e] = (unsigned long long)__double_as_longlong(q);
        p.max_ratio = fmax(p.max_ratio, q);
        if (q > 1.0) p.n_fail++;
        if (isfinite((double)c) && isfinite(r)) {
            const double df = (double)c - r;
            p.sum_sq_diff += df * df;
            p.sum_sq_ref += r * r;
        }
    }
    sp[threadIdx.x] = p;
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            Partial &a = sp[threadIdx.x];
            const Partial &b = sp[threadIdx.x + w];
            a.max_ratio = fmax(a.max_ratio, b.max_ratio);
            a.sum_sq_diff += b.sum_sq_diff;
            a.sum_sq_ref += b.sum_sq_ref;
            a.n_fail += b.n_fail;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sp[0];
}

__global__ void __launch_bounds__(RT)
err_fold_kernel(const Partial *__restrict__ part, int nparts, Partial *__restrict__ out,
                SelectState *__restrict__ st, unsigned long long rank,
                unsigned long long *__restrict__ hist) {
    __shared__ Partial sp[RT];
    Partial p{0.0, 0.0, 0.0, 0ull};
    for (int b = threadIdx.x; b < nparts; b += RT) {
        const Partial &q = part[b];
        p.max_ratio = fmax(p.max_ratio, q.max_ratio);
        p.sum_sq_diff += q.sum_sq_diff;
        p.sum_sq_ref += q.sum_sq_ref;
        p.n_fail += q.n_fail;
    }
    sp[threadIdx.x] = p;
    hist[threadIdx.x] = 0ull;
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            Partial &a = sp[threadIdx.x];
            const Partial &b = sp[threadIdx.x + w];
            a.max_ratio = fmax(a.max_ratio, b.max_ratio);
            a.sum_sq_diff += b.sum_sq_diff;
            a.sum_sq_ref += b.sum_sq_ref;
            a.n_fail += b.n_fail;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = sp[0];
        st->prefix = 0ull;
        st->mask = 0ull;
        st->rank = rank;
    }
}

__global__ void __launch_bounds__(RT)
radix_hist_kernel(const unsigned long long *__restrict__ keys, int64_t total,
                  const SelectState *__restrict__ st, int shift,
                  unsigned long long *__restrict__ hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    for (int64_t e = (int64_t)blockIdx.x * RT + threadIdx.x; e < total; e += (int64_t)gridDim.x * RT) {
        const unsigned long long k = keys[e];
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255ull], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void radix_pick_kernel(SelectState *__restrict__ st, int shift,
                                  unsigned long long *__restrict__ hist) {
    if (threadIdx.x != 0) return;
    unsigned long long rank = st->rank, cum = 0ull;
    int digit = 255;
    for (int d = 0; d < 256; ++d) {
        if (cum + hist[d] > rank) { digit = d; break; }
        cum += hist[d];
    }
    st->rank = rank - cum;
    st->prefix |= (unsigned long long)digit << shift;
    st->mask |= 255ull << shift;
    for (int d = 0; d < 256; ++d) hist[d] = 0ull;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t err_report_ws(int64_t m, int64_t n) {
    const size_t total = (size_t)(m > 0 ? m : 0) * (size_t)(n > 0 ? n : 0);
    return align256(total * 8) + align256(sizeof(Partial) * 4096) + align256(sizeof(Partial)) +
           align256(sizeof(SelectState)) + align256(256 * 8);
}

cudaError_t run_err_report(int sm_count, int64_t m, int64_t n, int64_t k, const float *C,
                           int64_t ldc, const double *C64, int64_t ldc64, const double *D,
                           int64_t ldd, void *ws, gb_err_report_t *out, cudaStream_t s) {
    const int64_t total = m * n;
    char *w = static_cast<char *>(ws);
    auto *keys = reinterpret_cast<unsigned long long *>(w);
    w += align256((size_t)total * 8);
    auto *part = reinterpret_cast<Partial *>(w);
    w += align256(sizeof(Partial) * 4096);
    auto *fin = reinterpret_cast<Partial *>(w);
    w += align256(sizeof(Partial));
    auto *st = reinterpret_cast<SelectState *>(w);
    w += align256(sizeof(SelectState));
    auto *hist = reinterpret_cast<unsigned long long *>(w);

    int blocks = sm_count * 4;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    const double kfac = 2.0 * (double)(k > 1 ? k : 1) * 0x1p-24;
    err_ratio_kernel<<<blocks, RT, 0, s>>>(m, n, kfac, C, ldc, C64, ldc64, D, ldd, keys, part);
    const unsigned long long rank = total > 0 ? (unsigned long long)((total - 1) / 2) : 0ull;
    err_fold_kernel<<<1, RT, 0, s>>>(part, blocks, fin, st, rank, hist);
    for (int b = 7; b >= 0; --b) {
        radix_hist_kernel<<<blocks, RT, 0, s>>>(keys, total, st, 8 * b, hist);
        radix_pick_kernel<<<1, 32, 0, s>>>(st, 8 * b, hist);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Partial hp;
    SelectState hs;
    e = cudaMemcpyAsync(&hp, fin, sizeof(hp), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    out->max_ratio = hp.max_ratio;
    unsigned long long key = hs.prefix;
    double med;
    memcpy(&med, &key, sizeof(med));
    out->median_ratio = total > 0 ? med : 0.0;
    out->sum_sq_diff = hp.sum_sq_diff;
    out->sum_sq_ref = hp.sum_sq_ref;
    out->n_fail = (int64_t)hp.n_fail;
    out->count = total;
    return cudaSuccess;
}

}  // namespace gb
