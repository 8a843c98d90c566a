// Host side of the C ABI declared in include/gbsgemm.h: argument checks in
// Level-3 BLAS order, quick returns, workspace layout, algorithm dispatch,
// the backward formulas and the device error word.
#include <stdlib.h>
#include <string.h>

#include <new>

#include "internal.h"

using namespace gb;

namespace {

bool trans_ok(char t) {
    return t == 'N' || t == 'n' || t == 'T' || t == 't' || t == 'C' || t == 'c';
}
bool is_trans(char t) { return t != 'N' && t != 'n'; }
int64_t max1(int64_t x) { return x > 1 ? x : 1; }

// BLAS xerbla positions: 1 transa, 2 transb, 3 M, 4 N, 5 K, 8 lda, 10 ldb, 13 ldc.
int check_sgemm_args(char ta, char tb, int64_t m, int64_t n, int64_t k, int64_t lda,
                     int64_t ldb, int64_t ldc) {
    if (!trans_ok(ta)) return -1;
    if (!trans_ok(tb)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (lda < max1(is_trans(ta) ? k : m)) return -8;
    if (ldb < max1(is_trans(tb) ? n : k)) return -10;
    if (ldc < max1(m)) return -13;
    return 0;
}

int check_handle(gb_handle_t h) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != h->device) return GB_ERR_HANDLE;
    return GB_OK;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of the terms of one packed operand (mn rows of op(A), or mn columns
// of op(B)): terms x mn x kpad elements, K contiguous.
size_t terms_bytes(int mode, bool a_side, int64_t mn, int64_t k) {
    return (size_t)split_parts_side(mode, a_side) * (size_t)split_kpad(mode, k) *
           (size_t)split_elem_bytes(mode) * (size_t)mn;
}

// Bytes of one packed operand: its terms, and for the scaled FP16 split the
// largest magnitude of each row after them (256-byte aligned, mn words).
size_t packed_bytes(int mode, bool a_side, int64_t mn, int64_t k) {
    const size_t t = terms_bytes(mode, a_side, mn, k);
    return mode == 4 ? round_up(t, 256) + (size_t)mn * sizeof(uint32_t) : t;
}

// The row maxima inside a packed operand of the scaled FP16 split.
uint32_t *packed_max(void *packed, int mode, bool a_side, int64_t mn, int64_t k) {
    return reinterpret_cast<uint32_t *>(static_cast<char *>(packed) +
                                        round_up(terms_bytes(mode, a_side, mn, k), 256));
}

// Workspace of the skinny kernel: [short operand packed][partial slots and
// tile counters], 1 KiB aligned.
size_t skinny_ws_total(int mode, int64_t m, int64_t n, int64_t k) {
    const bool xb = skinny_x_is_b(m, n);
    return round_up(packed_bytes(mode, xb, xb ? m : n, k), 1024) +
           round_up(skinny_ws_bytes(xb ? n : m), 1024);
}

// Workspace of a split algorithm: [A packed][B packed][split-K partials],
// each region 1 KiB aligned; the partials exist only when K is split. For a
// skinny shape, at least the skinny kernel's (which one runs depends on the
// operands' alignment, unknown here).
size_t split_ws_bytes(int mode, int64_t m, int64_t n, int64_t k) {
    const int s = split_k_factor(mode, m, n, k);
    const size_t partials = s > 1 ? (size_t)s * (size_t)m * (size_t)n * sizeof(float) : 0;
    const size_t two_pass = round_up(packed_bytes(mode, true, m, k), 1024) +
                            round_up(packed_bytes(mode, false, n, k), 1024) + round_up(partials, 1024);
    if (!skinny_shape(mode, m, n, k)) return two_pass;
    const size_t sk = skinny_ws_total(mode, m, n, k);
    return sk > two_pass ? sk : two_pass;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? GB_OK : GB_ERR_CUDA; }

}  // namespace

int gb::split_mode(gb_algo_t algo) {
    switch (algo) {
        case GB_ALGO_SPLIT_TF32X3: return 0;
        case GB_ALGO_SPLIT_BF16X3: return 1;
        case GB_ALGO_SPLIT_BF16X6: return 2;
        case GB_ALGO_SPLIT_BF16X9: return 3;
        case GB_ALGO_SPLIT_FP16X3: return 4;
        default: return -1;
    }
}

// AUTO picks the fastest algorithm whose worst-case error stays within the
// FP32 bound 2*K*u*D for this K. Each split drops a fixed relative term per
// product (BF16 x 2: 3*2^-16, BF16 x 3: 2*2^-24) and the tensor cores'
// accumulation adds up to one ulp per MMA instruction; requiring the dropped
// terms to use at most half of 2*K*u gives K >= 1024 for BF16 x 2, and the
// accumulation model K >= 9 for BF16 x 3 (which is also faster than TF32 x 2
// at the same accuracy class).
gb_algo_t gb::resolve_algo(gb_algo_t algo, int64_t k) {
    if (algo != GB_ALGO_AUTO) return algo;
    if (k >= 1024) return GB_ALGO_SPLIT_BF16X3;
    if (k >= kMinKBf16x6) return GB_ALGO_SPLIT_BF16X6;
    return GB_ALGO_SIMT;
}

// Split-K: when a problem has too few output tiles to occupy the GPU (at most
// 37 tiles of 128 x BN) and a long K (>= 1024), each tile's K range is cut
// into S slices so that about 148 work units run at once (S <= K/256, so a
// slice always holds several k-blocks, and S <= 16). Depends on the shape
// only: workspace sizes do not depend on the device.
int gb::split_k_factor(int mode, int64_t m, int64_t n, int64_t k) {
    const int64_t bn = tc_tile_n(mode, tc_rb128(mode, m, n, k));   // the kernel's tile width
    const int64_t tiles = ((m + 127) / 128) * ((n + bn - 1) / bn);
    if (tiles < 1 || tiles * 4 > 148 || k < 1024) return 1;
    int64_t s = 148 / tiles;
    if (s > k / 256) s = k / 256;
    if (s > 16) s = 16;
    return s > 1 ? (int)s : 1;
}

namespace {

// Split + pack one operand. a_side: op(A) (element (i,p) = op(A)[i,p]);
// else op(B)^T (element (j,p) = op(B)[p,j]).
cudaError_t pack_operand(int mode, bool a_side, bool trans, int64_t mn, int64_t k,
                         const float *X, int64_t ldx, void *out, cudaStream_t s) {
    const int64_t kpad = split_kpad(mode, k);
    // op(A): stored A is K-contiguous iff transposed; op(B)^T: stored B is
    // K-contiguous iff NOT transposed.
    const bool kcontig = a_side ? trans : !trans;
    if (mode == 4)
        return launch_split_pack_fp16(a_side, kcontig, mn, k, X, ldx, out, kpad, mn * kpad,
                                      packed_max(out, mode, a_side, mn, k), s);
    return launch_split_pack(mode, kcontig, mn, k, X, ldx, out, kpad, mn * kpad, s);
}

int compute_packed(gb_handle_t h, int mode, int64_t m, int64_t n, int64_t k, float alpha,
                   const void *Ap, const void *Bp, float beta, float *C, int64_t ldc,
                   cudaStream_t s, float *part = nullptr, int splits = 1,
                   const EpiOp *epi = nullptr) {
    const int64_t kpad = split_kpad(mode, k);
    TcArgs t{};
    t.mode = mode;
    t.m = m; t.n = n; t.k = k; t.kpad = kpad;
    t.alpha = alpha; t.beta = beta;
    t.Ap = Ap; t.Bp = Bp;
    t.a_part_stride = m * kpad; t.b_part_stride = n * kpad;
    t.C = C; t.ldc = ldc;
    t.part = part;
    t.splits = part ? splits : 1;
    t.dstate = h->dstate;
    t.wait_limit = h->wait_limit;
    t.sm_count = h->sm_count;
    t.row_bytes = h->rb_override ? h->rb_override : tuned_row_bytes(h, mode, m, n, k);
    if (epi) t.epi = *epi;
    if (mode == 4) {
        t.amax = packed_max(const_cast<void *>(Ap), mode, true, m, k);
        t.bmax = packed_max(const_cast<void *>(Bp), mode, false, n, k);
    }
    if (h->promote_k > 0) {
        const int64_t bk = tc_promo_kblock(mode);
        const int64_t kb = (h->promote_k + bk - 1) / bk;
        t.promote_kb = (int)(kb < 1 ? 1 : kb > (1 << 24) ? (1 << 24) : kb);
    }
    cudaError_t e = launch_tc_sgemm(t, s);
    return e == cudaSuccess ? GB_OK : (e == cudaErrorNotSupported ? GB_ERR_UNSUPPORTED : GB_ERR_CUDA);
}

}  // namespace

size_t gb::packed_operand_bytes(int mode, bool a_side, int64_t mn, int64_t k) {
    return packed_bytes(mode, a_side, mn, k);
}

// The product of a row range of a packed op(A) and a column range of a
// packed op(B) (see internal.h).
int gb::compute_packed_view(gb_handle_t h, int mode, int64_t m, int64_t n, int64_t k,
                            float alpha, const void *Ap, int64_t a_rows, int64_t a_row0,
                            const void *Bp, int64_t b_rows, int64_t b_row0, float beta, float *C,
                            int64_t ldc, cudaStream_t s, int64_t k0, int64_t kstride) {
    if (mode == 4 && (b_row0 % 256) != 0) return GB_ERR_ARG;   // one scaling block per tile
    if (mode == 4 && (k0 != 0 || kstride != 0)) return GB_ERR_ARG;   // maxima are per whole row
    const int64_t kpad = kstride > 0 ? kstride : split_kpad(mode, k);
    const int64_t eb = split_elem_bytes(mode);
    // TMA needs 16-byte aligned rows: the row stride and the K offset in
    // whole 16-byte groups (the packing pads rows to that)
    if (kpad < k0 + k || (kpad * eb) % 16 != 0 || (k0 * eb) % 16 != 0) return GB_ERR_ARG;
    TcArgs t{};
    t.mode = mode;
    t.m = m; t.n = n; t.k = k; t.kpad = kpad;
    t.alpha = alpha; t.beta = beta;
    t.Ap = static_cast<const char *>(Ap) + (a_row0 * kpad + k0) * eb;
    t.Bp = static_cast<const char *>(Bp) + (b_row0 * kpad + k0) * eb;
    t.a_part_stride = a_rows * kpad; t.b_part_stride = b_rows * kpad;
    t.C = C; t.ldc = ldc;
    t.splits = 1;
    t.dstate = h->dstate;
    t.wait_limit = h->wait_limit;
    t.sm_count = h->sm_count;
    if (mode == 4) {
        t.amax = packed_max(const_cast<void *>(Ap), mode, true, a_rows, k) + a_row0;
        t.bmax = packed_max(const_cast<void *>(Bp), mode, false, b_rows, k) + b_row0 / 256;
    }
    if (h->promote_k > 0) {
        const int64_t bk = tc_promo_kblock(mode);
        const int64_t kb = (h->promote_k + bk - 1) / bk;
        t.promote_kb = (int)(kb < 1 ? 1 : kb > (1 << 24) ? (1 << 24) : kb);
    }
    cudaError_t e = launch_tc_sgemm(t, s);
    return e == cudaSuccess ? GB_OK : (e == cudaErrorNotSupported ? GB_ERR_UNSUPPORTED : GB_ERR_CUDA);
}

// Splits and packs rows [row0, row0 + rows) of op(X) into their place in a
// packed operand of total_rows rows (terms total_rows * kpad apart); for the
// scaled FP16 split also their row maxima.
cudaError_t gb::pack_operand_rows(int mode, bool a_side, bool trans, int64_t rows, int64_t k,
                                  const float *X, int64_t ldx, void *packed, int64_t total_rows,
                                  int64_t row0, cudaStream_t s) {
    const int64_t kpad = split_kpad(mode, k);
    const bool kcontig = a_side ? trans : !trans;
    char *out = static_cast<char *>(packed) + row0 * kpad * split_elem_bytes(mode);
    if (mode == 4) {
        if (!a_side && (row0 % 256) != 0) return cudaErrorInvalidValue;
        uint32_t *mx = packed_max(packed, mode, a_side, total_rows, k) + (a_side ? row0 : row0 / 256);
        return launch_split_pack_fp16(a_side, kcontig, rows, k, X, ldx, out, kpad,
                                      total_rows * kpad, mx, s);
    }
    return launch_split_pack(mode, kcontig, rows, k, X, ldx, out, kpad, total_rows * kpad, s);
}

namespace {

int sgemm_impl(gb_handle_t h, gb_algo_t algo, char ta, char tb, int64_t m, int64_t n, int64_t k,
               float alpha, const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
               float *C, int64_t ldc, void *ws, size_t ws_bytes, cudaStream_t s) {
    int rc = check_sgemm_args(ta, tb, m, n, k, lda, ldb, ldc);
    if (rc) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if ((rc = check_handle(h))) return rc;
    if (m == 0 || n == 0 || ((alpha == 0.f || k == 0) && beta == 1.f)) return GB_OK;
    if (!C) return GB_ERR_ARG;
    if (alpha == 0.f || k == 0) return cuda_status(launch_scale_c(m, n, beta, C, ldc, s));
    if (!A || !B) return GB_ERR_ARG;

    algo = resolve_algo(algo, k);
    if (algo == GB_ALGO_SIMT) {
        SimtArgs a{is_trans(ta), is_trans(tb), m, n, k, alpha, beta, A, lda, B, ldb, C, ldc};
        return cuda_status(launch_simt_sgemm(a, s));
    }
    const int mode = split_mode(algo);
    const size_t need = split_ws_bytes(mode, m, n, k);
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return GB_ERR_WORKSPACE;
    char *Ap = static_cast<char *>(ws);
    char *Bp = Ap + round_up(packed_bytes(mode, true, m, k), 1024);
    char *Pp = Bp + round_up(packed_bytes(mode, false, n, k), 1024);
    const int splits = split_k_factor(mode, m, n, k);
    // A skinny product whose long operand TMA can read in place: split that
    // operand inside the kernel (one pass over it), pack only the short one.
    if (h->skinny_split && h->promote_k == 0 && skinny_supported(mode, m, n, k, A, lda, B, ldb)) {
        SkinnyArgs g{};
        g.mode = mode;
        g.ta = is_trans(ta); g.tb = is_trans(tb);
        g.x_is_b = skinny_x_is_b(m, n);
        g.m = m; g.n = n; g.k = k;
        g.alpha = alpha; g.beta = beta;
        g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
        g.C = C; g.ldc = ldc;
        g.kpad = split_kpad(mode, k);
        char *Yp = static_cast<char *>(ws);
        const int64_t yrows = g.x_is_b ? m : n;
        g.Yp = Yp;
        g.ws = Yp + round_up(packed_bytes(mode, g.x_is_b, yrows, k), 1024);
        g.dstate = h->dstate;
        g.wait_limit = h->wait_limit;
        g.sm_count = h->sm_count;
        cudaError_t e = skinny_clear(g, s);
        if (e == cudaSuccess)
            e = g.x_is_b ? pack_operand(mode, true, g.ta, m, k, A, lda, Yp, s)
                         : pack_operand(mode, false, g.tb, n, k, B, ldb, Yp, s);
        if (e == cudaSuccess) e = launch_tc_skinny(g, s);
        if (e != cudaErrorNotSupported) return cuda_status(e);
    }
    // Split fused into the tensor-core kernel, when the handle allows it and
    // TMA can read A and B as they are; otherwise the separate split/pack
    // pass. For K > 2048 both give bit-identical results.
    if (h->fused_split && h->promote_k == 0 && fused_supported(mode, A, lda, B, ldb, m, n, k)) {
        FusedArgs f{};
        f.mode = mode;
        f.ta = is_trans(ta); f.tb = is_trans(tb);
        f.m = m; f.n = n; f.k = k;
        f.alpha = alpha; f.beta = beta;
        f.A = A; f.lda = lda; f.B = B; f.ldb = ldb;
        f.C = C; f.ldc = ldc;
        f.part = splits > 1 ? reinterpret_cast<float *>(Pp) : nullptr;
        f.splits = splits;
        f.dstate = h->dstate;
        f.wait_limit = h->wait_limit;
        f.sm_count = h->sm_count;
        cudaError_t fe = launch_tc_fused(f, s);
        if (fe == cudaSuccess) return GB_OK;
        if (fe != cudaErrorNotSupported) return GB_ERR_CUDA;
    }
    cudaError_t e = pack_operand(mode, true, is_trans(ta), m, k, A, lda, Ap, s);
    if (e == cudaSuccess) e = pack_operand(mode, false, is_trans(tb), n, k, B, ldb, Bp, s);
    if (e != cudaSuccess) return GB_ERR_CUDA;
    return compute_packed(h, mode, m, n, k, alpha, Ap, Bp, beta, C, ldc, s,
                          splits > 1 ? reinterpret_cast<float *>(Pp) : nullptr, splits);
}

}  // namespace

int gb::sgemm_epi(gb_handle_t h, gb_algo_t algo, char ta, char tb, int64_t m, int64_t n,
                  int64_t k, float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                  float beta, float *C, int64_t ldc, const EpiOp &op, void *ws, size_t ws_bytes,
                  cudaStream_t s, bool *fused) {
    *fused = false;
    int rc = check_sgemm_args(ta, tb, m, n, k, lda, ldb, ldc);
    if (rc) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if ((rc = check_handle(h))) return rc;
    const int mode = (alpha == 0.f || k == 0) ? -1 : split_mode(resolve_algo(algo, k));
    const bool can_fuse = op.kind != 0 && m > 0 && n > 0 && A && B && C && (mode == 1 || mode == 2) &&
                          split_k_factor(mode, m, n, k) == 1 && h->promote_k == 0;
    if (!can_fuse)
        return sgemm_impl(h, algo, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws,
                          ws_bytes, s);
    const size_t need = split_ws_bytes(mode, m, n, k);
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return GB_ERR_WORKSPACE;
    char *Ap = static_cast<char *>(ws);
    char *Bp = Ap + round_up(packed_bytes(mode, true, m, k), 1024);
    cudaError_t e = pack_operand(mode, true, is_trans(ta), m, k, A, lda, Ap, s);
    if (e == cudaSuccess) e = pack_operand(mode, false, is_trans(tb), n, k, B, ldb, Bp, s);
    if (e != cudaSuccess) return GB_ERR_CUDA;
    rc = compute_packed(h, mode, m, n, k, alpha, Ap, Bp, beta, C, ldc, s, nullptr, 1, &op);
    if (rc == GB_OK) *fused = true;
    return rc;
}

namespace {

// Backward products (see gb_sgemm_backward in the header for the formulas).
struct BwdCall {
    char ta, tb;
    int64_t m, n, k;
    const float *A; int64_t lda;
    const float *B; int64_t ldb;
    float *C; int64_t ldc;
};

BwdCall grad_a(char ta, char tb, int64_t m, int64_t n, int64_t k, const float *B, int64_t ldb,
               const float *G, int64_t ldg, float *dA, int64_t ldda) {
    if (!is_trans(ta))   // dA (M x K) = G (M x N) * op(B)^T (N x K)
        return BwdCall{'N', is_trans(tb) ? 'N' : 'T', m, k, n, G, ldg, B, ldb, dA, ldda};
    // dA (K x M) = op(B) (K x N) * G^T (N x M)
    return BwdCall{is_trans(tb) ? 'T' : 'N', 'T', k, m, n, B, ldb, G, ldg, dA, ldda};
}

BwdCall grad_b(char ta, char tb, int64_t m, int64_t n, int64_t k, const float *A, int64_t lda,
               const float *G, int64_t ldg, float *dB, int64_t lddb) {
    if (!is_trans(tb))   // dB (K x N) = op(A)^T (K x M) * G (M x N)
        return BwdCall{is_trans(ta) ? 'N' : 'T', 'N', k, n, m, A, lda, G, ldg, dB, lddb};
    // dB (N x K) = G^T (N x M) * op(A) (M x K)
    return BwdCall{'T', is_trans(ta) ? 'T' : 'N', n, k, m, G, ldg, A, lda, dB, lddb};
}

size_t call_ws(gb_algo_t algo, const BwdCall &c) {
    algo = resolve_algo(algo, c.k);
    const int mode = split_mode(algo);
    return mode < 0 ? 0 : split_ws_bytes(mode, c.m, c.n, c.k);
}

}  // namespace

extern "C" {

GB_API int gb_version(void) { return 10000; }

GB_API const char *gb_status_string(int status) {
    if (status < 0) return "invalid SGEMM argument (negative code = BLAS argument position)";
    switch (status) {
        case GB_OK: return "success";
        case GB_ERR_CUDA: return "CUDA error";
        case GB_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case GB_ERR_UNSUPPORTED: return "unsupported device or request";
        case GB_ERR_TIMEOUT: return "bounded device wait expired";
        case GB_ERR_PLAN: return "invalid grouped plan";
        case GB_ERR_HANDLE: return "invalid handle or wrong current device";
        case GB_ERR_ARG: return "invalid argument";
        default: return "unknown status";
    }
}

GB_API int gb_create(gb_handle_t *out) {
    if (!out) return GB_ERR_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return GB_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return GB_ERR_UNSUPPORTED;
    gb_handle_s *h = new (std::nothrow) gb_handle_s();
    if (!h) return GB_ERR_ARG;
    h->magic = kHandleMagic;
    h->device = dev;
    h->sm_count = prop.multiProcessorCount;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    h->wait_limit = 2000000;
    h->skinny_split = true;
    strncpy(h->gpu_name, prop.name, sizeof(h->gpu_name) - 1);
    if (cudaRuntimeGetVersion(&h->cuda_runtime_version) != cudaSuccess) h->cuda_runtime_version = 0;
    if (cudaMalloc(&h->dstate, sizeof(DeviceState)) != cudaSuccess ||
        cudaMemset(h->dstate, 0, sizeof(DeviceState)) != cudaSuccess) {
        delete h;
        return GB_ERR_CUDA;
    }
    // gb_sgemm_noalloc's scratch array: looked up here, at set-up, so that it
    // is reserved on this device now and its calls never load anything.
    if (gb::noalloc_scratch_lookup(&h->noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->dstate);
        delete h;
        return GB_ERR_CUDA;
    }
    gb::tuning_autoload(h);
    *out = h;
    return GB_OK;
}

GB_API int gb_destroy(gb_handle_t h) {
    if (!h) return GB_OK;
    if (h->magic != kHandleMagic) return GB_ERR_HANDLE;
    cudaDeviceSynchronize();
    gb::destroy_pipe(h);
    gb::destroy_side(h);
    gb::destroy_trsm_graph(h);
    cudaFree(h->dstate);
    h->magic = 0;
    delete h;
    return GB_OK;
}

GB_API int gb_sgemm_workspace_size(gb_algo_t algo, char ta, char tb, int64_t m, int64_t n,
                                   int64_t k, size_t *bytes) {
    int rc = check_sgemm_args(ta, tb, m, n, k, max1(is_trans(ta) ? k : m),
                              max1(is_trans(tb) ? n : k), max1(m));
    if (rc) return rc;
    if (!bytes) return GB_ERR_ARG;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    const int mode = split_mode(resolve_algo(algo, k));
    *bytes = (mode < 0 || m == 0 || n == 0 || k == 0) ? 0 : split_ws_bytes(mode, m, n, k);
    return GB_OK;
}

GB_API int gb_sgemm(gb_handle_t h, gb_algo_t algo, char transa, char transb, int64_t m, int64_t n,
                    int64_t k, float alpha, const float *A, int64_t lda, const float *B,
                    int64_t ldb, float beta, float *C, int64_t ldc, void *workspace,
                    size_t ws_bytes, void *stream) {
    return sgemm_impl(h, algo, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                      workspace, ws_bytes, static_cast<cudaStream_t>(stream));
}

GB_API int gb_sgemm_pack_size(gb_algo_t algo, char which, int64_t mn, int64_t k, size_t *bytes) {
    if (which != 'A' && which != 'a' && which != 'B' && which != 'b') return -1;
    if (mn < 0) return -3;
    if (k < 0) return -5;
    if (!bytes) return GB_ERR_ARG;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    const int mode = split_mode(resolve_algo(algo, k));
    if (mode < 0) return GB_ERR_UNSUPPORTED;
    *bytes = packed_bytes(mode, which == 'A' || which == 'a', mn, k);
    return GB_OK;
}

GB_API int gb_sgemm_pack(gb_handle_t h, gb_algo_t algo, char which, char trans, int64_t mn,
                         int64_t k, const float *X, int64_t ldx, void *packed, size_t bytes,
                         void *stream) {
    const bool a_side = which == 'A' || which == 'a';
    if (!a_side && which != 'B' && which != 'b') return -1;
    if (!trans_ok(trans)) return -1;
    if (mn < 0) return -3;
    if (k < 0) return -5;
    // stored rows: op(A) = A is M x K, A^T stored K x M; op(B) = B is K x N, B^T stored N x K
    const int64_t rows = a_side ? (is_trans(trans) ? k : mn) : (is_trans(trans) ? mn : k);
    if (ldx < max1(rows)) return -8;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    int rc = check_handle(h);
    if (rc) return rc;
    const int mode = split_mode(resolve_algo(algo, k));
    if (mode < 0) return GB_ERR_UNSUPPORTED;
    if (mn == 0 || k == 0) return GB_OK;
    if (!X) return GB_ERR_ARG;
    if (!packed || bytes < packed_bytes(mode, a_side, mn, k) ||
        (reinterpret_cast<uintptr_t>(packed) & 255))
        return GB_ERR_WORKSPACE;
    return cuda_status(pack_operand(mode, a_side, is_trans(trans), mn, k, X, ldx, packed,
                                    static_cast<cudaStream_t>(stream)));
}

GB_API int gb_sgemm_compute(gb_handle_t h, gb_algo_t algo, int64_t m, int64_t n, int64_t k,
                            float alpha, const void *Apacked, const void *Bpacked, float beta,
                            float *C, int64_t ldc, void *stream) {
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (ldc < max1(m)) return -13;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    int rc = check_handle(h);
    if (rc) return rc;
    const int mode = split_mode(resolve_algo(algo, k));
    if (mode < 0) return GB_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m == 0 || n == 0 || ((alpha == 0.f || k == 0) && beta == 1.f)) return GB_OK;
    if (!C) return GB_ERR_ARG;
    if (alpha == 0.f || k == 0) return cuda_status(launch_scale_c(m, n, beta, C, ldc, s));
    if (!Apacked || !Bpacked || (reinterpret_cast<uintptr_t>(Apacked) & 255) ||
        (reinterpret_cast<uintptr_t>(Bpacked) & 255))
        return GB_ERR_WORKSPACE;
    return compute_packed(h, mode, m, n, k, alpha, Apacked, Bpacked, beta, C, ldc, s);
}

GB_API int gb_sgemm_backward_workspace_size(gb_algo_t algo, char ta, char tb, int64_t m,
                                            int64_t n, int64_t k, size_t *bytes) {
    int rc = check_sgemm_args(ta, tb, m, n, k, max1(is_trans(ta) ? k : m),
                              max1(is_trans(tb) ? n : k), max1(m));
    if (rc) return rc;
    if (!bytes) return GB_ERR_ARG;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if (m == 0 || n == 0 || k == 0) { *bytes = 0; return GB_OK; }
    const BwdCall a = grad_a(ta, tb, m, n, k, nullptr, 1, nullptr, 1, nullptr, 1);
    const BwdCall b = grad_b(ta, tb, m, n, k, nullptr, 1, nullptr, 1, nullptr, 1);
    const size_t wa = call_ws(algo, a), wb = call_ws(algo, b);
    *bytes = wa > wb ? wa : wb;
    return GB_OK;
}

GB_API int gb_sgemm_backward(gb_handle_t h, gb_algo_t algo, char ta, char tb, int64_t m,
                             int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
                             const float *B, int64_t ldb, float beta, const float *dC,
                             int64_t lddc, float *dA, int64_t ldda, float *dB, int64_t lddb,
                             float *dCin, int64_t lddcin, void *ws, size_t ws_bytes,
                             void *stream) {
    int rc = check_sgemm_args(ta, tb, m, n, k, lda, ldb, lddc);
    if (rc) return rc;
    if ((rc = check_handle(h))) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if (dA && ldda < max1(is_trans(ta) ? k : m)) return GB_ERR_ARG;
    if (dB && lddb < max1(is_trans(tb) ? n : k)) return GB_ERR_ARG;
    if (dCin && lddcin < max1(m)) return GB_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dA) {
        const BwdCall c = grad_a(ta, tb, m, n, k, B, ldb, dC, lddc, dA, ldda);
        rc = sgemm_impl(h, algo, c.ta, c.tb, c.m, c.n, c.k, alpha, c.A, c.lda, c.B, c.ldb, 0.f,
                        c.C, c.ldc, ws, ws_bytes, s);
        if (rc) return rc;
    }
    if (dB) {
        const BwdCall c = grad_b(ta, tb, m, n, k, A, lda, dC, lddc, dB, lddb);
        rc = sgemm_impl(h, algo, c.ta, c.tb, c.m, c.n, c.k, alpha, c.A, c.lda, c.B, c.ldb, 0.f,
                        c.C, c.ldc, ws, ws_bytes, s);
        if (rc) return rc;
    }
    if (dCin && m > 0 && n > 0) {
        if (beta != 0.f && !dC) return GB_ERR_ARG;
        rc = cuda_status(launch_scaled_copy(m, n, beta, dC, lddc, dCin, lddcin, s));
        if (rc) return rc;
    }
    return GB_OK;
}

GB_API size_t gb_err_report_workspace_size(int64_t m, int64_t n) {
    return err_report_ws(m, n);
}

GB_API int gb_err_report(gb_handle_t h, int64_t m, int64_t n, int64_t k, const float *C,
                         int64_t ldc, const double *C64, int64_t ldc64, const double *D,
                         int64_t ldd, void *ws, size_t ws_bytes, gb_err_report_t *out,
                         void *stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out || m < 0 || n < 0 || k < 0) return GB_ERR_ARG;
    if (ldc < max1(m) || ldc64 < max1(m) || ldd < max1(m)) return GB_ERR_ARG;
    if (m > 0 && n > 0 && (!C || !C64 || !D)) return GB_ERR_ARG;
    if (!ws || ws_bytes < err_report_ws(m, n) || (reinterpret_cast<uintptr_t>(ws) & 255))
        return GB_ERR_WORKSPACE;
    return cuda_status(run_err_report(h->sm_count, m, n, k, C, ldc, C64, ldc64, D, ldd, ws, out,
                                      static_cast<cudaStream_t>(stream)));
}

GB_API int gb_get_device_error(gb_handle_t h, void *stream, int *site) {
    int rc = check_handle(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int err[2] = {0, 0};
    if (cudaStreamSynchronize(s) != cudaSuccess) return GB_ERR_CUDA;
    if (cudaMemcpy(err, h->dstate->err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GB_ERR_CUDA;
    if (cudaMemset(h->dstate->err, 0, sizeof(err)) != cudaSuccess) return GB_ERR_CUDA;
    if (site) *site = (int)err[0];
    return err[1] ? GB_ERR_TIMEOUT : GB_OK;
}

GB_API int gb_set_fused_split(gb_handle_t h, int enable) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    h->fused_split = enable != 0;
    return GB_OK;
}

GB_API int gb_set_skinny_split(gb_handle_t h, int enable) {
    int rc = check_handle(h);
    if (rc) return rc;
    h->skinny_split = enable != 0;
    return GB_OK;
}

GB_API int gb_get_skinny_split(gb_handle_t h, int *enable) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!enable) return GB_ERR_ARG;
    *enable = h->skinny_split ? 1 : 0;
    return GB_OK;
}

GB_API int gb_set_promotion(gb_handle_t h, int64_t k_chunk) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    if (k_chunk < 0) return GB_ERR_ARG;
    h->promote_k = k_chunk;
    return GB_OK;
}

GB_API int gb_get_promotion(gb_handle_t h, int64_t *k_chunk) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    if (!k_chunk) return GB_ERR_ARG;
    *k_chunk = h->promote_k;
    return GB_OK;
}

GB_API int gb_set_wait_limit(gb_handle_t h, int64_t polls) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    if (polls < 1) return GB_ERR_ARG;
    h->wait_limit = polls;
    return GB_OK;
}

}  // extern "C"
