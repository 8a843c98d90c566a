// SSYRK on the tensor cores: C <- alpha op(A) op(A)^T + beta C on one
// triangle of C, in ONE persistent tcgen05 launch over that triangle's tiles.
//
// op(A) is split and packed once (the same K-major [terms][n][kpad] layout as
// an SGEMM operand); both MMA operands read that one buffer through two
// tensor maps (box heights 128 and BN). The work source enumerates only the
// 128 x BN tiles that meet the triangle, row of tiles by row of tiles, and
// the epilogue stores only the triangle's elements of the tiles the
// diagonal crosses (C is read only there, and only when beta != 0).
#include "tc_body.cuh"

namespace gb {
namespace {

using namespace tcx;

// The tiles (tm, tn) of an n x n output meeting its lower (tn*BN <= last row
// of the tile) or upper (last column >= first row) triangle, in row-major
// order. With R = BN / BM, tile row t holds floor(t/R) + 1 lower tiles or
// NT - floor(t/R) upper ones; the prefix counts have closed forms, and a
// unit's tile row is found by binary search over them.
template <int BN, int BK>
struct TriSource {
    static constexpr bool kTri = true;
    static constexpr int kEpi = 0;
    static constexpr int R = BN / BM;
    const CUtensorMap *ma, *mb;
    int64_t n;
    float alpha, beta;
    float *C;
    int64_t ldc;
    bool lower;
    int TM, NT, nkb;
    // number of tiles in tile rows 0 .. t-1
    __device__ __forceinline__ int64_t prefix(int t) const {
        const int64_t p = t / 2;
        const int64_t s = R == 1 ? (int64_t)t * (t - 1) / 2 : ((t & 1) ? p * p : p * (p - 1));
        return lower ? (int64_t)t + s : (int64_t)t * NT - s;
    }
    __device__ __forceinline__ int64_t num_units() const { return prefix(TM); }
    __device__ __forceinline__ void unit(int64_t u, UnitInfo &ui) const {
        int lo = 0, hi = TM;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix(mid) <= u) lo = mid; else hi = mid;
        }
        const int64_t o = u - prefix(lo);
        ui.tm = lo;
        ui.tn = lower ? o : (int64_t)(lo / R) + o;
        ui.kb0 = 0;
        ui.kb1 = nkb;
        ui.ma = ma; ui.mb = mb;
        ui.M = n; ui.N = n;
        ui.alpha = alpha; ui.beta = beta;
        ui.raw = false;
        ui.dst = C;
        ui.ldd = ldc;
        ui.lower = lower;
    }
};

template <int MODE, int RB>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_syrk_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               int64_t n, int64_t k, float alpha, float beta, float *__restrict__ C, int64_t ldc,
               int lower, DeviceState *dstate, uint64_t limit_ns) {
    using CF = Cfg<MODE, RB>;
    if (threadIdx.x == 0) {
        prefetch_tmap(&mapA);
        prefetch_tmap(&mapB);
    }
    TriSource<CF::BN, CF::BK> src;
    src.ma = &mapA; src.mb = &mapB;
    src.n = n;
    src.alpha = alpha; src.beta = beta;
    src.C = C; src.ldc = ldc;
    src.lower = lower != 0;
    src.TM = (int)((n + BM - 1) / BM);
    src.NT = (int)((n + CF::BN - 1) / CF::BN);
    src.nkb = (int)((k + CF::BK - 1) / CF::BK);
    tc_body<MODE, RB>(src, dstate, limit_ns);
}

template <int MODE, int RB>
cudaError_t launch_syrk_mode(const TcSyrkArgs &a, cudaStream_t s) {
    using CF = Cfg<MODE, RB>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_syrk_kernel<MODE, RB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    if (a.n > (int64_t)1 << 30 || a.k > 2147483647LL) return cudaErrorNotSupported;
    alignas(64) CUtensorMap ma, mb;
    if (!tc_make_operand_map(&ma, MODE, RB == 128, a.packed, a.k, a.n, true) ||
        !tc_make_operand_map(&mb, MODE, RB == 128, a.packed, a.k, a.n, false))
        return cudaErrorInvalidValue;
    // the work source's tile count (its prefix formula at t = TM)
    const int64_t TM = (a.n + BM - 1) / BM, NT = (a.n + CF::BN - 1) / CF::BN, p = TM / 2;
    const int64_t fl = CF::BN == BM ? TM * (TM - 1) / 2 : ((TM & 1) ? p * p : p * (p - 1));
    const int64_t units = a.lower ? TM + fl : TM * NT - fl;
    int grid = a.sm_count > 0 ? a.sm_count : 1;
    if (units < grid) grid = (int)units;
    tc_syrk_kernel<MODE, RB><<<grid, NUM_THREADS, CF::SMEM_BYTES, s>>>(
        ma, mb, a.n, a.k, a.alpha, a.beta, a.C, a.ldc, a.lower ? 1 : 0, a.dstate,
        (uint64_t)a.wait_limit * 1000ull);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_syrk(const TcSyrkArgs &a, cudaStream_t s) {
    const bool rb128 = tc_rb128(a.mode, a.n, a.n, a.k);   // the one-GEMM kernel's row width rule
    switch (a.mode) {
        case 0: return rb128 ? launch_syrk_mode<0, 128>(a, s) : launch_syrk_mode<0, 64>(a, s);
        case 1: return rb128 ? launch_syrk_mode<1, 128>(a, s) : launch_syrk_mode<1, 64>(a, s);
        case 2: return rb128 ? launch_syrk_mode<2, 128>(a, s) : launch_syrk_mode<2, 64>(a, s);
        case 3: return rb128 ? launch_syrk_mode<3, 128>(a, s) : launch_syrk_mode<3, 64>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
