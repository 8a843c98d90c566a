// gb_sgemm_host: C <- alpha op(A) op(B) + beta C with A, B, C in host memory.
//
// The copies over the host link are overlapped with the GEMM: op(A) is copied
// once (and, for the split algorithms, split and packed once); op(B) and C are
// streamed in blocks of columns through two device slots. Three of the
// handle's own streams form the pipeline
//     copy-in   B_j (and C_j when beta != 0) -> slot j % 2      ev_in
//     compute   pack B_j, GEMM of block j into slot j % 2       ev_done
//     copy-out  C_j -> host                                    ev_out
// so the upload of block j+1, the GEMM of block j and the download of block
// j-1 run at once; a slot is refilled only after its download finished. The
// pipeline starts after the work already enqueued on the caller's stream and
// the caller's stream waits for its last download, so the call is ordered on
// that stream like any other, and returns without waiting.
#include <stdint.h>

#include "internal.h"

namespace gb {
namespace {

bool is_t(char c) { return c == 'T' || c == 't' || c == 'C' || c == 'c'; }
bool trans_ok(char c) { return is_t(c) || c == 'N' || c == 'n'; }
int64_t max1(int64_t x) { return x > 1 ? x : 1; }
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Columns per block: about an eighth of N (at least 256, a multiple of 128),
// so that eight or more blocks keep the three stages busy. Shape-only.
int64_t block_cols(int64_t n) {
    int64_t nb = (n + 7) / 8;
    nb = (nb + 127) / 128 * 128;
    if (nb < 256) nb = 256;
    return nb < n ? nb : n;
}

struct Layout {
    int mode;                 // split mode, -1 for SIMT
    bool compute;             // false: C <- beta C only (alpha = 0 or K = 0)
    int64_t nb;
    size_t a_dev, a_pack, b_dev, b_pack, c_dev;     // byte offsets (slot 0 for B and C)
    size_t slot;                                    // bytes between the two slots
    size_t total;
};

int layout(gb_algo_t algo, char ta, char tb, int64_t m, int64_t n, int64_t k, float alpha,
           Layout *L) {
    L->compute = !(alpha == 0.f || k == 0);
    L->mode = L->compute ? split_mode(resolve_algo(algo, k)) : -1;
    L->nb = block_cols(n);
    const size_t a_bytes = L->compute ? (size_t)m * (size_t)k * 4 : 0;
    size_t a_pack = 0, b_pack = 0;
    if (L->mode >= 0) {
        if (gb_sgemm_pack_size(algo, 'A', m, k, &a_pack) || gb_sgemm_pack_size(algo, 'B', L->nb, k, &b_pack))
            return GB_ERR_ARG;
    }
    L->a_dev = 0;
    L->a_pack = round_up(a_bytes, 256);
    L->b_dev = L->a_pack + round_up(a_pack, 256);
    const size_t b_bytes = L->compute ? (size_t)k * (size_t)L->nb * 4 : 0;
    L->b_pack = L->b_dev + round_up(b_bytes, 256);
    L->c_dev = L->b_pack + round_up(b_pack, 256);
    const size_t c_bytes = (size_t)m * (size_t)L->nb * 4;
    L->slot = L->c_dev + round_up(c_bytes, 256) - L->b_dev;
    L->total = L->b_dev + 2 * L->slot;
    (void)ta; (void)tb;
    return GB_OK;
}

int check_args(char ta, char tb, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
               int64_t ldc) {
    if (!trans_ok(ta)) return -1;
    if (!trans_ok(tb)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (lda < max1(is_t(ta) ? k : m)) return -8;
    if (ldb < max1(is_t(tb) ? n : k)) return -10;
    if (ldc < max1(m)) return -13;
    return GB_OK;
}

// The handle's pipeline streams and events, created on first use.
bool pipe_ready(gb_handle_t h) {
    if (h->pipe_ready) return true;
    for (int i = 0; i < 3; ++i)
        if (cudaStreamCreateWithFlags(&h->pipe_stream[i], cudaStreamNonBlocking) != cudaSuccess)
            return false;
    for (int i = 0; i < kPipeEvents; ++i)
        if (cudaEventCreateWithFlags(&h->pipe_event[i], cudaEventDisableTiming) != cudaSuccess)
            return false;
    h->pipe_ready = true;
    return true;
}

}  // namespace

void destroy_pipe(gb_handle_t h) {
    if (!h->pipe_ready) return;
    for (int i = 0; i < 3; ++i) cudaStreamDestroy(h->pipe_stream[i]);
    for (int i = 0; i < kPipeEvents; ++i) cudaEventDestroy(h->pipe_event[i]);
    h->pipe_ready = false;
}

}  // namespace gb

extern "C" {

GB_API int gb_sgemm_host_workspace_size(gb_algo_t algo, char ta, char tb, int64_t m, int64_t n,
                                        int64_t k, size_t *bytes) {
    using namespace gb;
    int rc = check_args(ta, tb, m, n, k, max1(is_t(ta) ? k : m), max1(is_t(tb) ? n : k), max1(m));
    if (rc) return rc;
    if (!bytes || algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if (m == 0 || n == 0) { *bytes = 0; return GB_OK; }
    Layout L;
    rc = layout(algo, ta, tb, m, n, k, 1.f, &L);
    if (rc) return rc;
    *bytes = L.total;
    return GB_OK;
}

GB_API int gb_sgemm_host(gb_handle_t h, gb_algo_t algo, char ta, char tb, int64_t m, int64_t n,
                         int64_t k, float alpha, const float *A, int64_t lda, const float *B,
                         int64_t ldb, float beta, float *C, int64_t ldc, void *workspace,
                         size_t ws_bytes, void *stream) {
    using namespace gb;
    int rc = check_args(ta, tb, m, n, k, lda, ldb, ldc);
    if (rc) return rc;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != h->device) return GB_ERR_HANDLE;
    if (m == 0 || n == 0 || ((alpha == 0.f || k == 0) && beta == 1.f)) return GB_OK;
    Layout L;
    rc = layout(algo, ta, tb, m, n, k, alpha, &L);
    if (rc) return rc;
    if (!C || (L.compute && (!A || !B))) return GB_ERR_ARG;
    size_t full = 0;
    gb_sgemm_host_workspace_size(algo, ta, tb, m, n, k, &full);
    if (ws_bytes < full || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return GB_ERR_WORKSPACE;
    if (!pipe_ready(h)) return GB_ERR_CUDA;

    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t sin = h->pipe_stream[0], scomp = h->pipe_stream[1], sout = h->pipe_stream[2];
    cudaEvent_t *ev = h->pipe_event;
    cudaEvent_t ev_start = ev[0], ev_a = ev[1];
    cudaEvent_t ev_in[2] = {ev[2], ev[3]}, ev_done[2] = {ev[4], ev[5]}, ev_out[2] = {ev[6], ev[7]};
    char *ws = static_cast<char *>(workspace);
    float *Ad = reinterpret_cast<float *>(ws + L.a_dev);
    void *Ap = ws + L.a_pack;
    const int64_t rows_a = is_t(ta) ? k : m, cols_a = is_t(ta) ? m : k;
    const bool tb_t = is_t(tb);
    const bool read_c = beta != 0.f;
    const size_t pb = L.mode >= 0 ? L.c_dev - L.b_pack : 0;     // packed B slot bytes

#define GB_TRY(x) do { if ((x) != cudaSuccess) return GB_ERR_CUDA; } while (0)
    GB_TRY(cudaEventRecord(ev_start, user));
    for (int i = 0; i < 3; ++i) GB_TRY(cudaStreamWaitEvent(h->pipe_stream[i], ev_start, 0));
    if (L.compute) {
        GB_TRY(cudaMemcpy2DAsync(Ad, (size_t)rows_a * 4, A, (size_t)lda * 4, (size_t)rows_a * 4,
                                 (size_t)cols_a, cudaMemcpyHostToDevice, sin));
        GB_TRY(cudaEventRecord(ev_a, sin));
        GB_TRY(cudaStreamWaitEvent(scomp, ev_a, 0));
        if (L.mode >= 0) {
            size_t ap_bytes = 0;
            gb_sgemm_pack_size(algo, 'A', m, k, &ap_bytes);
            rc = gb_sgemm_pack(h, algo, 'A', ta, m, k, Ad, rows_a, Ap, ap_bytes, scomp);
            if (rc) return rc;
        }
    }
    const int64_t nblocks = (n + L.nb - 1) / L.nb;
    for (int64_t j = 0; j < nblocks; ++j) {
        const int sl = (int)(j & 1);
        const int64_t j0 = j * L.nb, nbj = (n - j0 < L.nb) ? n - j0 : L.nb;
        char *slot = ws + L.b_dev + (size_t)sl * L.slot;
        float *Bd = reinterpret_cast<float *>(slot);
        void *Bp = slot + (L.b_pack - L.b_dev);
        float *Cd = reinterpret_cast<float *>(slot + (L.c_dev - L.b_dev));
        // copy-in (the slot is free once block j - 2 has been downloaded)
        if (j >= 2) GB_TRY(cudaStreamWaitEvent(sin, ev_out[sl], 0));
        int64_t ldbd = 0;
        if (L.compute) {
            if (!tb_t) {        // op(B) block = columns j0.. of the k x n stored B
                ldbd = k;
                GB_TRY(cudaMemcpy2DAsync(Bd, (size_t)k * 4, B + j0 * ldb, (size_t)ldb * 4,
                                         (size_t)k * 4, (size_t)nbj, cudaMemcpyHostToDevice, sin));
            } else {            // rows j0.. of the n x k stored B
                ldbd = nbj;
                GB_TRY(cudaMemcpy2DAsync(Bd, (size_t)nbj * 4, B + j0, (size_t)ldb * 4,
                                         (size_t)nbj * 4, (size_t)k, cudaMemcpyHostToDevice, sin));
            }
        }
        if (read_c)
            GB_TRY(cudaMemcpy2DAsync(Cd, (size_t)m * 4, C + j0 * ldc, (size_t)ldc * 4, (size_t)m * 4,
                                     (size_t)nbj, cudaMemcpyHostToDevice, sin));
        GB_TRY(cudaEventRecord(ev_in[sl], sin));
        // compute
        GB_TRY(cudaStreamWaitEvent(scomp, ev_in[sl], 0));
        if (!L.compute) {
            GB_TRY(launch_scale_c(m, nbj, beta, Cd, m, scomp));
        } else if (L.mode >= 0) {
            rc = gb_sgemm_pack(h, algo, 'B', tb, nbj, k, Bd, ldbd, Bp, pb, scomp);
            if (!rc) rc = gb_sgemm_compute(h, algo, m, nbj, k, alpha, Ap, Bp, beta, Cd, m, scomp);
            if (rc) return rc;
        } else {
            rc = gb_sgemm(h, GB_ALGO_SIMT, ta, tb, m, nbj, k, alpha, Ad, rows_a, Bd, ldbd, beta,
                          Cd, m, nullptr, 0, scomp);
            if (rc) return rc;
        }
        GB_TRY(cudaEventRecord(ev_done[sl], scomp));
        // copy-out
        GB_TRY(cudaStreamWaitEvent(sout, ev_done[sl], 0));
        GB_TRY(cudaMemcpy2DAsync(C + j0 * ldc, (size_t)ldc * 4, Cd, (size_t)m * 4, (size_t)m * 4,
                                 (size_t)nbj, cudaMemcpyDeviceToHost, sout));
        GB_TRY(cudaEventRecord(ev_out[sl], sout));
    }
    for (int sl = 0; sl < 2 && sl < nblocks; ++sl) GB_TRY(cudaStreamWaitEvent(user, ev_out[sl], 0));
#undef GB_TRY
    return GB_OK;
}

}  // extern "C"
