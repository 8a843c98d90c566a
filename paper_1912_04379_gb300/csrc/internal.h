// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (see include/gbsgemm.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbsgemm.h"

namespace gb {

// Site ids written to the device error word when a bounded wait expires.
enum WaitSite : int {
    kSiteProducerEmpty = 1,   // TMA producer waiting for a free smem stage
    kSiteMmaFull = 2,         // MMA issuer waiting for a filled smem stage
    kSiteMmaAccEmpty = 3,     // MMA issuer waiting for the epilogue to drain TMEM
    kSiteEpiAccFull = 4,      // epilogue waiting for a finished accumulator
    kSiteTmemAlloc = 5,       // TMEM allocation did not complete
    kSiteDrain = 6,           // final drain of in-flight copies
    kSiteConvert = 7          // split converter waiting for an FP32 tile or a free operand stage
};

// Device error word layout: err[0] = first failing site (0 = none),
// err[1] = number of failures since the last read.
struct DeviceState {
    unsigned int err[2];
    unsigned int pad[62];
};

}  // namespace gb

struct gb_handle_s {
    int magic;
    int device;
    int sm_count;
    int cc_major, cc_minor;
    size_t smem_optin;
    int64_t wait_limit;
    gb::DeviceState *dstate;   // device memory
    // Grouped autotuner result, per size class of a problem (see grouped.cu):
    // 0 = SIMT 64x64 tiles, 1 = SIMT 128x128 tiles, 2 + v = tensor cores in
    // grouped configuration v.
    bool grouped_tuned;
    int grouped_choice[8];
    // the key of the tuning record, and the one-GEMM row widths measured per
    // shape bucket (gb_tune_sgemm); rb_override forces a width while tuning
    char gpu_name[96];
    int cuda_runtime_version;
    int n_gemm_rb;
    gb_tuning_gemm_t gemm_rb[GB_TUNING_MAX_GEMM];
    int rb_override;
    bool fused_split;           // allow the split fused into the tensor-core kernel (off by default)
    bool skinny_split;          // allow the skinny-product kernel (on by default)
    int64_t promote_k;          // promoted accumulation: chunk length in K (0 = off)
    // gb_sgemm_host's pipeline (copy-in, compute, copy-out), created on first use
    bool pipe_ready;
    cudaStream_t pipe_stream[6];   // copy-in, compute, copy-out, then pack and a second GEMM stream
    cudaEvent_t pipe_event[56];
    // grouped runs: a side stream for the SIMT part, forked from and joined
    // to the caller's stream (created when a plan has both parts)
    bool side_ready;
    cudaStream_t side_stream;
    cudaEvent_t side_event[2];
    // device address of gb_sgemm_noalloc's static scratch array on this
    // handle's device, looked up by gb_create (null if that failed)
    void *noalloc_scratch;
    // gb_strsm's last call as an instantiated CUDA graph with its arguments
    // (blas3.cu), replayed while the arguments repeat; created on first use
    void *trsm_graph;
};

namespace gb {

// Frees gb_strsm's cached graph (gb_destroy).
void destroy_trsm_graph(gb_handle_t h);

constexpr int kHandleMagic = 0x6b5e3a21;
// Smallest K at which each split meets the plain FP32 bound 2*K*u*D under the
// tensor-core accumulation model (each MMA instruction, 16 exact products or
// 8 for TF32 plus the running sum, errs by at most one FP32 ulp; derivation in
// gb_algo_t's comment in include/gbsgemm.h): BF16 x 3 terms with 6 products
// from K = 9, with all 9 products from K = 10, TF32 x 2 from K = 16 (its
// dropped terms), BF16 x 2 from K = 1024 (its dropped terms, using at most
// half the bound).
constexpr int64_t kMinKBf16x6 = 9;
constexpr int64_t kMinKBf16x9 = 10;
constexpr int kPipeStreams = 6;
constexpr int kPipeEvents = 56;   // 8 for the column-block pipeline, 48 for the 2-D one
void destroy_pipe(gb_handle_t h);     // releases gb_sgemm_host's streams and events
void destroy_side(gb_handle_t h);     // releases the grouped runs' side stream and events
// Device address of gb_sgemm_noalloc's static scratch array on the current
// device (loads the module that holds it, which reserves the array there).
cudaError_t noalloc_scratch_lookup(void **addr);

// ------------------------------------------------------------------ SIMT --
struct SimtArgs {
    bool ta, tb;                // true = transposed
    int64_t m, n, k;
    float alpha, beta;
    const float *A; int64_t lda;
    const float *B; int64_t ldb;
    float *C; int64_t ldc;
};
cudaError_t launch_simt_sgemm(const SimtArgs &a, cudaStream_t s);

// C <- beta*C (beta == 0 writes zeros without reading C).
cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float *C, int64_t ldc,
                           cudaStream_t s);

// Y <- beta*X elementwise (M x N; beta == 0 writes zeros without reading X).
cudaError_t launch_scaled_copy(int64_t m, int64_t n, float beta, const float *X, int64_t ldx,
                               float *Y, int64_t ldy, cudaStream_t s);

// ------------------------------------------------------ split/pack pass --
// Splits op(X) (rows x k; rows = M for A, N for B^T) into `parts` terms and
// writes each term as a row-major [rows][kpad] array (K contiguous).
// kcontig: the stored matrix is K-contiguous (element (r,p) at X[p + r*ld]),
// else rows-contiguous (element (r,p) at X[r + p*ld]).
// mode: 0 = TF32 (4-byte words, 2 parts), 1 = BF16 2 parts, 2 and 3 = BF16 3 parts
// (the tensor-core kernel then forms 6 or all 9 products of the terms).
cudaError_t launch_split_pack(int mode, bool kcontig, int64_t rows, int64_t k,
                              const float *X, int64_t ld, void *out, int64_t kpad,
                              int64_t part_stride_elems, cudaStream_t s);
// Mode 4 (the scaled FP16 split, FP16X3): first mx[r] = the largest finite
// |x| of row r (FP32 bits), then the terms of each row scaled by its power of
// two: op(A) rows (a_side) as 3 terms (2^11 h, h, l), op(B)^T rows as 2 (h, l).
cudaError_t launch_split_pack_fp16(bool a_side, bool kcontig, int64_t rows, int64_t k,
                                   const float *X, int64_t ld, void *out, int64_t kpad,
                                   int64_t part_stride_elems, uint32_t *mx, cudaStream_t s);

// -------------------------------------------------- tensor-core kernel ---
// Elementwise operation fused into the tensor-core epilogue, applied to
// v = alpha*acc + beta*C at output element (i, j) before it is stored:
//   kind 1: v <- act(v + bias[i])    (act = tanh or the identity)
//   kind 2: v <- v * (1 - aux_ij^2)  (aux: M x N column-major, ld = ldaux)
struct EpiOp {
    int kind = 0;
    int tanh_act = 0;
    const float *bias = nullptr;
    const float *aux = nullptr;
    int64_t ldaux = 0;
};

struct TcArgs {
    int mode;                   // as launch_split_pack
    int64_t m, n, k, kpad;
    float alpha, beta;
    const void *Ap;             // [parts][m][kpad]
    const void *Bp;             // [parts][n][kpad]
    int64_t a_part_stride, b_part_stride;   // elements between parts
    float *C; int64_t ldc;
    float *part;                // split-K partial sums (splits x m x n floats) or null
    int splits;                 // K slices per output tile (1 = no split)
    DeviceState *dstate;
    int64_t wait_limit;
    int sm_count;
    EpiOp epi;                  // kind != 0: BF16 x 2 or x 3 terms, no split-K
    int promote_kb;             // > 0: promoted accumulation, k-blocks per chunk
    const uint32_t *amax;       // mode 4: largest |op(A)| per row (FP32 bits)
    const uint32_t *bmax;       // mode 4: largest |op(B)| per column
    int row_bytes;              // 64 or 128: the tuned row width; 0: the built-in rule
};
// cudaErrorNotSupported: an epilogue operation with another mode or split-K,
// or with promoted accumulation.
cudaError_t launch_tc_sgemm(const TcArgs &a, cudaStream_t s);
// Elements of K in one k-block of the promoted-accumulation kernel (its
// chunks are whole k-blocks): 16 for TF32 terms, 32 for BF16 terms.
int tc_promo_kblock(int mode);
// Number of K slices gb_sgemm uses for a split-precision problem (depends on
// the shape only, so workspace sizes do not depend on the device).
int split_k_factor(int mode, int64_t m, int64_t n, int64_t k);
// C = alpha * (sum of S split-K partials, in slice order) + beta * C.
cudaError_t launch_splitk_reduce(int64_t m, int64_t n, int S, const float *part, float alpha,
                                 float beta, float *C, int64_t ldc, cudaStream_t s);

// ------------------------------------------ split fused into the kernel --
struct FusedArgs {
    int mode;                   // 1 = BF16 x 2 terms, 2 = BF16 x 3 terms
    bool ta, tb;
    int64_t m, n, k;
    float alpha, beta;
    const float *A; int64_t lda;
    const float *B; int64_t ldb;
    float *C; int64_t ldc;
    float *part;                // split-K partials (splits x m x n floats) or null
    int splits;
    DeviceState *dstate;
    int64_t wait_limit;
    int sm_count;
};
// True when the caller's A and B can be read by TMA directly (16-byte
// aligned, leading dimensions multiples of 4) for a BF16 split mode.
bool fused_supported(int mode, const float *A, int64_t lda, const float *B, int64_t ldb,
                     int64_t m, int64_t n, int64_t k);
// Split-precision SGEMM reading FP32 operands directly (no pack pass).
// cudaErrorNotSupported: use the two-pass path instead.
cudaError_t launch_tc_fused(const FusedArgs &a, cudaStream_t s);
// ------------------------------------ skinny products, split in the kernel --
// One operand (Y) has at most 64 rows, the other (X) is long: X is read as
// FP32 by TMA and split inside the kernel, Y is packed beforehand.
constexpr int kSkinnyMaxCtas = 256;   // the grid never exceeds this (workspace bound)
struct SkinnyArgs {
    int mode;                   // 1 = BF16 x 2 terms, 2 = x 3 terms (6 products), 3 = (9 products)
    bool ta, tb;
    bool x_is_b;                // X = op(B)^T (M short), else X = op(A) (N short)
    int64_t m, n, k;
    float alpha, beta;
    const float *A; int64_t lda;
    const float *B; int64_t ldb;
    const void *Yp;             // Y packed by launch_split_pack, terms Yrows * kpad apart
    int64_t kpad;
    float *C; int64_t ldc;
    void *ws;                   // skinny_ws_bytes(rows of X), 256-byte aligned
    DeviceState *dstate;
    int64_t wait_limit;
    int sm_count;
};
// Shapes the skinny kernel takes (a BF16 split, one side <= 64 rows, K >= 256
// and a long X).
bool skinny_shape(int mode, int64_t m, int64_t n, int64_t k);
bool skinny_x_is_b(int64_t m, int64_t n);
// skinny_shape, and TMA can read X in place (16-byte aligned, leading
// dimension a multiple of 4).
bool skinny_supported(int mode, int64_t m, int64_t n, int64_t k, const float *A, int64_t lda,
                      const float *B, int64_t ldb);
// Partial-sum slots and per-tile counters for X with R rows.
size_t skinny_ws_bytes(int64_t R);
// Zeroes the per-tile counters in a.ws; call before the pack of Y, which
// the kernel's launch then follows directly (it may overlap the pack's tail).
cudaError_t skinny_clear(const SkinnyArgs &a, cudaStream_t s);
// cudaErrorNotSupported: use the two-pass path instead.
cudaError_t launch_tc_skinny(const SkinnyArgs &a, cudaStream_t s);
// Workspace layout helpers shared by the API and the launcher.
int64_t split_kpad(int mode, int64_t k);
int split_parts(int mode);
int split_parts_side(int mode, bool a_side);   // mode 4: 3 terms for op(A), 2 for op(B)
int split_elem_bytes(int mode);

// ------------------------------------------------ grouped tensor-core path --
// One problem of a grouped tensor-core launch (device memory). Its operands
// were split and packed by launch_split_pack_grouped into buffers owned by
// the plan; mapA / mapB are their tensor maps, also in device memory.
struct TcProblem {
    const CUtensorMap *mapA;
    const CUtensorMap *mapB;
    float *C;
    int64_t ldc;
    int64_t m, n, k;
    float alpha, beta;
};
struct TcItem {
    int prob;
    int tm, tn;                 // output tile (128 x tile_n)
    int pad;
};
int tc_tile_n(int mode, bool rb128);
// Row width (128 bytes or 64) of the one-GEMM tensor-core kernel for a shape.
bool tc_rb128(int mode, int64_t m, int64_t n, int64_t k);
// Tensor map of one packed operand ([terms][rows][kpad], K innermost) for the
// kernel variant (mode, 128-byte rows or not); a_side selects the box height.
bool tc_make_operand_map(CUtensorMap *map, int mode, bool rb128, const void *packed, int64_t k,
                         int64_t rows, bool a_side);
// The grouped kernel's tile width (128 for every split) and operand maps.
// Grouped configurations v = 0..kGroupedConfigVariants-1 (see tc_body.cuh).
constexpr int kGroupedConfigVariants = 3;
int tc_grouped_tile_n(int v);
int tc_grouped_row_bytes(int v);
bool tc_make_grouped_operand_map(CUtensorMap *map, int mode, int v, const void *packed, int64_t k,
                                 int64_t rows, bool a_side);
cudaError_t launch_tc_grouped(int mode, int v, const TcProblem *probs, const TcItem *items,
                              int64_t nitems, int sm_count, DeviceState *dstate,
                              int64_t wait_limit, cudaStream_t s);

// SSYRK on the tensor cores: C <- alpha op(A) op(A)^T + beta C on one
// triangle, op(A) (n x k) already split and packed like an SGEMM A operand.
struct TcSyrkArgs {
    int mode;                   // as launch_split_pack
    const void *packed;         // [parts][n][kpad]
    int64_t n, k;
    float alpha, beta;
    float *C;
    int64_t ldc;
    bool lower;
    int sm_count;
    DeviceState *dstate;
    int64_t wait_limit;         // microseconds
};
cudaError_t launch_tc_syrk(const TcSyrkArgs &a, cudaStream_t s);

// gb_sgemm followed by the elementwise operation `op` fused into the
// tensor-core epilogue when the resolved algorithm is BF16 x 2 or x 3 terms
// and K is not split (*fused = true); otherwise plain gb_sgemm, and the
// caller applies `op` itself (*fused = false). Same workspace as gb_sgemm.
int sgemm_epi(gb_handle_t h, gb_algo_t algo, char ta, char tb, int64_t m, int64_t n, int64_t k,
              float alpha, const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
              float *C, int64_t ldc, const EpiOp &op, void *ws, size_t ws_bytes, cudaStream_t s,
              bool *fused);

// C <- alpha op(A)[a_row0 .. a_row0+m) op(B)[:, b_row0 .. b_row0+n) + beta C,
// from whole packed operands of a_rows rows (op(A)) and b_rows columns
// (op(B)), as gb_sgemm_pack laid them out; no split-K. Mode 4 needs b_row0 a
// multiple of 256 (its column-block scaling). k0 / kstride (0: none / the
// operand's own padded K) take a K range [k0, k0 + k) of operands packed
// with row stride kstride (the K offset and stride in whole 16-byte groups;
// not mode 4). Returns a GB_* status.
int compute_packed_view(gb_handle_t h, int mode, int64_t m, int64_t n, int64_t k, float alpha,
                        const void *Ap, int64_t a_rows, int64_t a_row0, const void *Bp,
                        int64_t b_rows, int64_t b_row0, float beta, float *C, int64_t ldc,
                        cudaStream_t s, int64_t k0 = 0, int64_t kstride = 0);
// Split + pack rows [row0, row0+rows) of op(X) (a_side) or op(B)^T into the
// packed operand of total_rows rows at `packed` (layout of gb_sgemm_pack).
cudaError_t pack_operand_rows(int mode, bool a_side, bool trans, int64_t rows, int64_t k,
                              const float *X, int64_t ldx, void *packed, int64_t total_rows,
                              int64_t row0, cudaStream_t s);
// Bytes of one packed operand (gb_sgemm_pack_size's value).
size_t packed_operand_bytes(int mode, bool a_side, int64_t mn, int64_t k);

// Tuning (tuning.cu, grouped.cu): the row width recorded for a call's shape
// bucket (0: none), the grouped autotuner, and the GB_SGEMM_TUNING cache.
int tuned_row_bytes(gb_handle_t h, int mode, int64_t m, int64_t n, int64_t k);
int grouped_autotune(gb_handle_t h);
void tuning_autosave(gb_handle_t h);
void tuning_autoload(gb_handle_t h);

// AUTO's choice for a given K, and the split mode of an algorithm (-1: SIMT).
gb_algo_t resolve_algo(gb_algo_t algo, int64_t k);
int split_mode(gb_algo_t algo);

// One 64 x 64 (rows x k) tile of the grouped split/pack pass.
struct PackItem {
    const float *X;
    int64_t ld;
    void *out;                  // terms at out + t*ps, row r at r*kpad
    int64_t kpad, ps;
    int64_t rows, k;
    int64_t r0, p0;
    int kc;                     // source contiguous along K
    int vec;                    // 16-byte loads allowed
    int mode;                   // as launch_split_pack
    int pad_;
};
cudaError_t launch_split_pack_grouped(const PackItem *items, int64_t nitems, cudaStream_t s);

// --------------------------------------------------------- error report --
size_t err_report_ws(int64_t m, int64_t n);
cudaError_t run_err_report(int sm_count, int64_t m, int64_t n, int64_t k, const float *C,
                           int64_t ldc, const double *C64, int64_t ldc64, const double *D,
                           int64_t ldd, void *ws, gb_err_report_t *out, cudaStream_t s);

}  // namespace gb
