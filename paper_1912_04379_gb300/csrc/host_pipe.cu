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
//
// For the split algorithms with M and N of at least 2048 a 2-D blocked
// pipeline replaces it, so that no GEMM waits for all of op(A): op(A) is cut
// into row blocks A_s and op(B) into column blocks B_s (multiples of 256,
// about an eighth of each), uploaded in the order A_0, B_0, A_1, B_1, ...
// and each split and packed once, in place, into whole packed operands.
// When pair s has arrived, the output blocks (r, j) with max(r, j) = s can
// be computed: two GEMMs on views of the packed operands (A_s times B_0..s,
// and A_0..s-1 times B_s), each on its own stream so that one's last,
// partial wave of tiles overlaps the other, and those blocks (one row strip
// and one column strip of C) download as each GEMM finishes, while pair s + 1
// uploads and, on a fifth stream, is split and packed.
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
    for (int i = 0; i < kPipeStreams; ++i)
        if (cudaStreamCreateWithFlags(&h->pipe_stream[i], cudaStreamNonBlocking) != cudaSuccess)
            return false;
    for (int i = 0; i < kPipeEvents; ++i)
        if (cudaEventCreateWithFlags(&h->pipe_event[i], cudaEventDisableTiming) != cudaSuccess)
            return false;
    h->pipe_ready = true;
    return true;
}

// ---------------------------------------------- 2-D blocked pipeline --
// Row blocks of op(A) and column blocks of op(B), multiples of 256 (the
// scaled FP16 split scales op(B) per 256 columns). A long dimension (at
// least 6144) gets blocks that shrink toward its end, about 1/4, 3/16,
// 5/32, 1/8, 3/32, 1/16, 1/16, 1/32, 1/32 of it: everything the last pair
// of blocks leaves to do (the GEMMs of its L and their downloads) starts
// only after the last upload, so the last blocks should be small, while the
// large first blocks keep the early GEMMs efficient. Shorter dimensions get
// about eighths, at least 1024. Fills off[0..count] with the boundaries and
// returns count (<= kMaxBlocks2d).
constexpr int kMaxBlocks2d = 9;
int schedule_2d(int64_t x, int64_t *off) {
    const int64_t units = (x + 255) / 256;
    int count = 0;
    off[0] = 0;
    if (units >= 24) {
        static const int w[kMaxBlocks2d] = {8, 6, 5, 4, 3, 2, 2, 1, 1};   // in 32nds
        int64_t used = 0;
        for (int i = 0; i < kMaxBlocks2d; ++i) {
            int64_t u = (units * w[i] + 16) / 32;
            if (u < 1) u = 1;
            if (i == kMaxBlocks2d - 1 || used + u > units) u = units - used;
            if (u <= 0) break;
            used += u;
            off[++count] = used * 256 < x ? used * 256 : x;
            if (used >= units) break;
        }
        return count;
    }
    int64_t b = (x + 7) / 8;
    b = (b + 255) / 256 * 256;
    if (b < 1024) b = 1024;
    for (int64_t r = 0; r < x; r += b) off[++count] = r + b < x ? r + b : x;
    return count;
}

bool use_2d(int mode, int64_t m, int64_t n, bool compute) {
    return compute && mode >= 0 && m >= 2048 && n >= 2048;
}

struct Grid2 {
    int mode;
    int ra, cb;               // number of op(A) row blocks and op(B) column blocks
    int64_t aoff[kMaxBlocks2d + 1], boff[kMaxBlocks2d + 1];   // their boundaries
    size_t a_dev, b_dev, a_pack, b_pack, c_dev, total;
};

void grid2(int mode, int64_t m, int64_t n, int64_t k, Grid2 *G) {
    G->mode = mode;
    G->ra = schedule_2d(m, G->aoff);
    G->cb = schedule_2d(n, G->boff);
    size_t off = 0;
    G->a_dev = off; off += round_up((size_t)m * (size_t)k * 4, 256);      // op(A) as stored
    G->b_dev = off; off += round_up((size_t)k * (size_t)n * 4, 256);      // op(B) as stored
    G->a_pack = off; off += round_up(packed_operand_bytes(mode, true, m, k), 256);
    G->b_pack = off; off += round_up(packed_operand_bytes(mode, false, n, k), 256);
    G->c_dev = off; off += round_up((size_t)m * (size_t)n * 4, 256);     // C, ld = M
    G->total = off;
}

int run_2d(gb_handle_t h, const Grid2 &G, char ta, char tb, int64_t m, int64_t n, int64_t k,
           float alpha, const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
           float *C, int64_t ldc, char *ws, cudaStream_t user) {
    cudaStream_t sin = h->pipe_stream[0], sg1 = h->pipe_stream[1], sout = h->pipe_stream[2];
    cudaStream_t spack = h->pipe_stream[3], sg2 = h->pipe_stream[4];
    cudaEvent_t *ev = h->pipe_event + 8;             // [0] start, then 5 per pair, then the end
    const int pairs = G.ra > G.cb ? G.ra : G.cb;
    if (2 + 5 * pairs > kPipeEvents - 8) return GB_ERR_UNSUPPORTED;
    const bool ta_t = is_t(ta), tb_t = is_t(tb);
    // device copies keep the stored layout: op(A) rows are stored columns
    // when transposed (ld K), else stored rows (ld M); likewise for op(B)
    const int64_t lda_d = ta_t ? k : m, ldb_d = tb_t ? n : k;
    float *Ad = reinterpret_cast<float *>(ws + G.a_dev);
    float *Bd = reinterpret_cast<float *>(ws + G.b_dev);
    void *Ap = ws + G.a_pack, *Bp = ws + G.b_pack;
    float *Cd = reinterpret_cast<float *>(ws + G.c_dev);
    const bool read_c = beta != 0.f;
#define GB_TRY(x) do { if ((x) != cudaSuccess) return GB_ERR_CUDA; } while (0)
    GB_TRY(cudaEventRecord(ev[0], user));
    for (int i = 0; i < 5; ++i) GB_TRY(cudaStreamWaitEvent(h->pipe_stream[i], ev[0], 0));
    // the C strips of pair s: rows [r0, r1) x columns [0, c1) and rows [0, r0) x [c0, c1)
    auto strips = [&](int s, int64_t &r0, int64_t &r1, int64_t &c0, int64_t &c1) {
        r0 = s < G.ra ? G.aoff[s] : m;
        r1 = s < G.ra ? G.aoff[s + 1] : m;
        c0 = s < G.cb ? G.boff[s] : n;
        c1 = s < G.cb ? G.boff[s + 1] : n;
    };
    auto copy_c = [&](bool up, int64_t i0, int64_t i1, int64_t j0, int64_t j1, cudaStream_t st) {
        if (i1 <= i0 || j1 <= j0) return cudaSuccess;
        return up ? cudaMemcpy2DAsync(Cd + i0 + j0 * m, (size_t)m * 4, C + i0 + j0 * ldc,
                                      (size_t)ldc * 4, (size_t)(i1 - i0) * 4, (size_t)(j1 - j0),
                                      cudaMemcpyHostToDevice, st)
                  : cudaMemcpy2DAsync(C + i0 + j0 * ldc, (size_t)ldc * 4, Cd + i0 + j0 * m,
                                      (size_t)m * 4, (size_t)(i1 - i0) * 4, (size_t)(j1 - j0),
                                      cudaMemcpyDeviceToHost, st);
    };
    for (int s = 0; s < pairs; ++s) {
        cudaEvent_t ev_a = ev[1 + 5 * s], ev_b = ev[2 + 5 * s], ev_p = ev[3 + 5 * s];
        cudaEvent_t ev_g1 = ev[4 + 5 * s], ev_g2 = ev[5 + 5 * s];
        int64_t r0, r1, c0, c1;
        strips(s, r0, r1, c0, c1);
        // ---- upload A_s, then B_s (and the C strips when beta != 0)
        if (s < G.ra) {
            if (!ta_t)       // rows r0..r1 of the m x k stored A
                GB_TRY(cudaMemcpy2DAsync(Ad + r0, (size_t)m * 4, A + r0, (size_t)lda * 4,
                                         (size_t)(r1 - r0) * 4, (size_t)k, cudaMemcpyHostToDevice, sin));
            else             // columns r0..r1 of the k x m stored A
                GB_TRY(cudaMemcpy2DAsync(Ad + r0 * k, (size_t)k * 4, A + r0 * lda, (size_t)lda * 4,
                                         (size_t)k * 4, (size_t)(r1 - r0), cudaMemcpyHostToDevice, sin));
        }
        GB_TRY(cudaEventRecord(ev_a, sin));
        if (s < G.cb) {
            if (!tb_t)       // columns c0..c1 of the k x n stored B
                GB_TRY(cudaMemcpy2DAsync(Bd + c0 * k, (size_t)k * 4, B + c0 * ldb, (size_t)ldb * 4,
                                         (size_t)k * 4, (size_t)(c1 - c0), cudaMemcpyHostToDevice, sin));
            else             // rows c0..c1 of the n x k stored B
                GB_TRY(cudaMemcpy2DAsync(Bd + c0, (size_t)n * 4, B + c0, (size_t)ldb * 4,
                                         (size_t)(c1 - c0) * 4, (size_t)k, cudaMemcpyHostToDevice, sin));
        }
        if (read_c) {
            GB_TRY(copy_c(true, r0, r1, 0, c1, sin));
            GB_TRY(copy_c(true, 0, r0, c0, c1, sin));
        }
        GB_TRY(cudaEventRecord(ev_b, sin));
        // ---- split and pack A_s and B_s in place (their own stream)
        GB_TRY(cudaStreamWaitEvent(spack, ev_a, 0));
        if (s < G.ra)
            GB_TRY(pack_operand_rows(G.mode, true, ta_t, r1 - r0, k, ta_t ? Ad + r0 * k : Ad + r0,
                                     lda_d, Ap, m, r0, spack));
        GB_TRY(cudaStreamWaitEvent(spack, ev_b, 0));
        if (s < G.cb)
            GB_TRY(pack_operand_rows(G.mode, false, tb_t, c1 - c0, k, tb_t ? Bd + c0 : Bd + c0 * k,
                                     ldb_d, Bp, n, c0, spack));
        GB_TRY(cudaEventRecord(ev_p, spack));
        // ---- the two GEMMs of the L, on two streams (packs of pairs <= s done)
        int rc = GB_OK;
        GB_TRY(cudaStreamWaitEvent(sg1, ev_p, 0));
        if (r1 > r0 && c1 > 0)       // A_s x B_0 .. B_s
            rc = compute_packed_view(h, G.mode, r1 - r0, c1, k, alpha, Ap, m, r0, Bp, n, 0, beta,
                                     Cd + r0, m, sg1);
        if (rc) return rc;
        GB_TRY(cudaEventRecord(ev_g1, sg1));
        GB_TRY(cudaStreamWaitEvent(sg2, ev_p, 0));
        if (r0 > 0 && c1 > c0)       // A_0 .. A_s-1 x B_s
            rc = compute_packed_view(h, G.mode, r0, c1 - c0, k, alpha, Ap, m, 0, Bp, n, c0, beta,
                                     Cd + c0 * m, m, sg2);
        if (rc) return rc;
        GB_TRY(cudaEventRecord(ev_g2, sg2));
        // ---- download each strip when its GEMM is done
        GB_TRY(cudaStreamWaitEvent(sout, ev_g1, 0));
        GB_TRY(copy_c(false, r0, r1, 0, c1, sout));
        GB_TRY(cudaStreamWaitEvent(sout, ev_g2, 0));
        GB_TRY(copy_c(false, 0, r0, c0, c1, sout));
    }
    cudaEvent_t ev_end = ev[1 + 5 * pairs];
    GB_TRY(cudaEventRecord(ev_end, sout));
    GB_TRY(cudaStreamWaitEvent(user, ev_end, 0));
#undef GB_TRY
    return GB_OK;
}

}  // namespace

void destroy_pipe(gb_handle_t h) {
    if (!h->pipe_ready) return;
    for (int i = 0; i < kPipeStreams; ++i) cudaStreamDestroy(h->pipe_stream[i]);
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
    if (use_2d(L.mode, m, n, L.compute)) {
        Grid2 G;
        grid2(L.mode, m, n, k, &G);
        *bytes = G.total;
    }
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
    if (use_2d(L.mode, m, n, L.compute)) {
        Grid2 G;
        grid2(L.mode, m, n, k, &G);
        return run_2d(h, G, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                      static_cast<char *>(workspace), static_cast<cudaStream_t>(stream));
    }

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
