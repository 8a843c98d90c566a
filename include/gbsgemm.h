/*
 * gbsgemm.h - C ABI of a GB300 (sm_103a) single-precision GEMM library.
 *
 * The operation is the Level-3 BLAS SGEMM (paper Sec. 1: dense product of
 * A: M x K and B: K x N costing 2MNK flops, exposed through the SGEMM
 * interface of Level-3 BLAS):
 *
 *     C <- alpha * op(A) * op(B) + beta * C
 *
 * op(X) = X for trans 'N'/'n' and X^T for 'T'/'t'/'C'/'c' (real data, so
 * 'C' equals 'T'). op(A) is M x K, op(B) is K x N, C is M x N. All matrices
 * are column-major: element (r,c) of X lives at X[r + c*ldX].
 *
 * Conventions for every entry point below
 * ---------------------------------------
 * - Pointers named A, B, C, dC, ... are DEVICE pointers on the handle's GPU;
 *   pointers to structs and sizes (gb_handle_t*, size_t*, gb_err_report_t*,
 *   host_problems) are HOST pointers. The caller owns every buffer, the
 *   workspace and the stream; the library never frees caller memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Compute calls enqueue work on it and return without waiting,
 *   unless their comment says they synchronise.
 * - Level-3 BLAS semantics: if beta == 0, C is not read (NaN there does not
 *   propagate); if alpha == 0 or K == 0, A and B are not read. Quick return
 *   (nothing enqueued) when M == 0, N == 0, or (alpha == 0 or K == 0) and
 *   beta == 1.
 * - Return codes: 0 = success. A negative code -i names the i-th SGEMM
 *   argument in BLAS order that is invalid (1 transa, 2 transb, 3 M, 4 N,
 *   5 K, 8 lda, 10 ldb, 13 ldc), as BLAS's xerbla would, but returned
 *   instead of aborting. Positive codes are the GB_ERR_* values below.
 *   Nothing is enqueued when a call returns an error before launching.
 * - Thread safety: a handle may be used from one host thread at a time.
 */
#ifndef GBSGEMM_H
#define GBSGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GB_API __attribute__((visibility("default")))
#else
#define GB_API
#endif

/* Status codes (positive); negative codes are BLAS argument positions. */
enum {
    GB_OK = 0,
    GB_ERR_CUDA = 1,        /* a CUDA runtime/driver call failed */
    GB_ERR_WORKSPACE = 2,   /* workspace NULL, misaligned or too small */
    GB_ERR_UNSUPPORTED = 3, /* device is not sm_103, or an unsupported request */
    GB_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (see gb_get_device_error) */
    GB_ERR_PLAN = 5,        /* invalid or mismatched grouped plan */
    GB_ERR_HANDLE = 6,      /* NULL or destroyed handle, or wrong current device */
    GB_ERR_ARG = 7          /* invalid argument outside the SGEMM list (NULL out-pointer, count < 0, ...) */
};

/* Algorithms. All compute C in FP32 storage; they differ in how the
 * products are formed:
 *  GB_ALGO_SIMT         FP32 fused multiply-add on the CUDA cores.
 *  GB_ALGO_SPLIT_TF32X3 each operand split as a = hi + lo, both TF32
 *                       (round to nearest even); hi*hi + hi*lo + lo*hi on
 *                       the tensor cores (tcgen05 kind::tf32), FP32 accumulation.
 *  GB_ALGO_SPLIT_BF16X3 hi/lo in BF16; the same three products (kind::f16).
 *  GB_ALGO_SPLIT_BF16X6 a = b0 + b1 + b2 in BF16 (exact for FP32 inputs);
 *                       the six products with weight >= 2^-16:
 *                       b0b0 b0b1 b1b0 b0b2 b1b1 b2b0.
 *  GB_ALGO_SPLIT_BF16X9 the same three BF16 terms and all nine products, so
 *                       every FP32 product a*b is formed exactly (each BF16
 *                       x BF16 product is exact in FP32); only the FP32
 *                       accumulation rounds. 1.5x the tensor work of BF16X6.
 *  GB_ALGO_SPLIT_FP16X3 each row of op(A) and each block of 256 columns of
 *                       op(B) is first scaled by a power of two (from its
 *                       largest finite magnitude, so that the FP16 terms stay
 *                       in range), then
 *                       split as x = h + l*2^-11, h and l FP16 (11 significant
 *                       bits each, round to nearest even); h*h + h*l + l*h on
 *                       the tensor cores (kind::f16) in one FP32 accumulator,
 *                       at the rate of BF16X3, with TF32X3's per-product
 *                       error; the scaling is undone exactly in the epilogue.
 *                       It always runs the promoted-accumulation kernel (see
 *                       gb_set_promotion; with promotion off, one chunk spans
 *                       K). Grouped runs and gb_ssyrk's triangle kernel take
 *                       SPLIT_TF32X3 for it.
 *  GB_ALGO_AUTO         the library picks: SPLIT_BF16X3 when K >= 1024,
 *                       SPLIT_BF16X6 when 9 <= K < 1024, else SIMT.
 * Error per element, D = |alpha||op(A)||op(B)| + |beta||C|, u = 2^-24:
 *  SIMT       |C - C_exact| <= 2*max(K,1)*u*D
 *  split x    (2*max(K,1)*u + e_x + t_x)*D, with e_x the dropped cross terms
 *             (TF32X3 and FP16X3 3*2^-22, BF16X3 3*2^-16, BF16X6 2*2^-24
 *             x 1.01, BF16X9 0) and t_x the tensor cores' accumulation.
 *             The PTX ISA leaves that accumulation's rounding unspecified
 *             (it is not round-to-nearest: BF16X9, whose products are all
 *             exact, measured 1.34 x 2*K*u*D at K = 1). The library assumes
 *             a model: every MMA instruction adds its 16 exact products (8
 *             for TF32) to the running sum with an error of at most one FP32
 *             ulp (2u relative). An element then sees P*ceil(K/16) such steps
 *             (P products per pair of terms: 3, 6 or 9; ceil(K/8) for TF32),
 *             plus one rounding in the alpha/beta epilogue, so
 *             (2*P*ceil(K/16) + 2)*u*D bounds accumulation and epilogue
 *             together. Against the plain bound 2*K*u*D this leaves room for
 *             the dropped terms once K >= 16 (TF32X3, FP16X3), 1024 (BF16X3,
 *             its dropped terms within half the bound), 9 (BF16X6) or 10
 *             (BF16X9); below that the model gives t_x = (2*P*ceil(K/16) +
 *             2 - 2*K)*u (BF16X9 at most 18u). AUTO and the grouped
 *             planner use a split only above its threshold.
 *  FP16X3     additionally |alpha|*2^-34*(2^(la_i - 3)*sum_p |b_pj|
 *             + 2^(lb_J - 14)*sum_p |a_ip|), la_i = floor(log2 max_p |a_ip|) and
 *             lb_J = floor(log2 of the largest |b_pl| over the block of 256
 *             columns l holding j) (finite entries; a = op(A), b = op(B)):
 *             the last term is what entries far below their row's or column
 *             block's largest magnitude lose (from about 2^-17 of it for
 *             op(A), 2^-28 for op(B), down to nothing below 2^-40).
 *             It is negligible when no such entries dominate an element's
 *             sum (M = N = K = 8192 with magnitudes 2^U(-20,20): largest
 *             error 0.0004 of the plain bound), but with few widely spread
 *             entries (K = 8, the same magnitudes) it can exceed the plain
 *             bound many times over. AUTO never picks FP16X3.
 *  The BF16 three-term split is exact for |a| >= 2^-110; smaller nonzero
 *  magnitudes lose bits below the BF16 subnormal range. */
typedef enum {
    GB_ALGO_AUTO = -1,
    GB_ALGO_SIMT = 0,
    GB_ALGO_SPLIT_TF32X3 = 1,
    GB_ALGO_SPLIT_BF16X3 = 2,
    GB_ALGO_SPLIT_BF16X6 = 3,
    GB_ALGO_SPLIT_BF16X9 = 4,
    GB_ALGO_SPLIT_FP16X3 = 5
} gb_algo_t;

typedef struct gb_handle_s *gb_handle_t;
typedef struct gb_grouped_plan_s *gb_grouped_plan_t;

/* Library version as 10000*major + 100*minor + patch. */
GB_API int gb_version(void);

/* Human-readable name of a status code (never NULL; static storage). */
GB_API const char *gb_status_string(int status);

/* Create a handle bound to the CURRENT CUDA device. Allocates a few hundred
 * bytes of device memory for the device error word and scratch counters,
 * and looks up the device address of gb_sgemm_noalloc's static scratch
 * array (the first handle on a device thereby reserves its 32 MiB).
 * Returns GB_ERR_UNSUPPORTED if the device is not compute capability 10.3,
 * GB_ERR_CUDA if no device is usable, GB_ERR_ARG if h is NULL. */
GB_API int gb_create(gb_handle_t *h);

/* Destroy a handle (synchronises the device first). NULL is a no-op. */
GB_API int gb_destroy(gb_handle_t h);

/* Bytes of device workspace gb_sgemm needs for this algorithm and problem
 * (0 for GB_ALGO_SIMT). Writes *bytes; returns a BLAS argument code on bad
 * arguments. The workspace pointer passed later must be 256-byte aligned. */
GB_API int gb_sgemm_workspace_size(gb_algo_t algo, char transa, char transb,
                                   int64_t m, int64_t n, int64_t k, size_t *bytes);

/* C <- alpha*op(A)*op(B) + beta*C (paper Sec. 1; Level-3 BLAS SGEMM).
 * Requirements: lda >= max(1, rows of stored A) (M if transa is 'N', else K),
 * ldb >= max(1, rows of stored B) (K if transb is 'N', else N),
 * ldc >= max(1, M). C must share no element with A or B (disjoint blocks of
 * one array are allowed). The split algorithms need
 * `workspace` of at least gb_sgemm_workspace_size() bytes, 256-byte aligned
 * (GB_ERR_WORKSPACE otherwise); SIMT ignores it. Enqueues on `stream` and
 * returns without waiting. A bounded-wait timeout inside a tensor-core
 * kernel is reported by gb_get_device_error, not by this call. The split
 * kernels choose their shared-memory row width (64 or 128 bytes of K per
 * row) by shape; the environment variable GB_SGEMM_TC_ROW_BYTES = 64 or 128,
 * read once per process, forces one of them (results stay within the same
 * bound; the order of the term products within a k-block differs). */
GB_API int gb_sgemm(gb_handle_t h, gb_algo_t algo, char transa, char transb,
                    int64_t m, int64_t n, int64_t k,
                    float alpha, const float *A, int64_t lda,
                    const float *B, int64_t ldb,
                    float beta, float *C, int64_t ldc,
                    void *workspace, size_t ws_bytes, void *stream);

/* gb_sgemm for callers that cannot allocate device memory. The paper has no
 * counterpart; this is a library convenience.
 *
 * Some callers can neither call cudaMalloc nor pass a workspace: plugins
 * inside a framework that owns all device memory through its own pool and
 * forbids raw allocations, latency-critical code that cannot take the
 * implicit synchronisation an allocation may cause, or processes whose
 * device memory is fully reserved. This entry point computes exactly what
 * gb_sgemm computes, with the same kernels and the same arguments minus the
 * workspace: the split workspace is a fixed array of GB_STATIC_SCRATCH_BYTES
 * (32 MiB) in device memory that belongs to the library, and the call
 * allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine). The caller still owns and passes A, B and C.
 * - The 32 MiB are reserved on a device when the first handle is created
 *   there (gb_create looks up the array's device address with that device
 *   current and keeps it in the handle) and stay reserved until the process
 *   exits. The call itself loads nothing and looks nothing up. A handle does
 *   not survive a reset of its device (cudaDeviceReset): create a new one.
 * - Returns GB_ERR_WORKSPACE, with nothing enqueued, when the problem's
 *   split workspace (gb_sgemm_workspace_size) is larger than
 *   GB_STATIC_SCRATCH_BYTES, e.g. BF16X3 fits M = N = K = 2048. SIMT needs
 *   no workspace and has no size limit here.
 * - All calls share the one array. Each call overwrites every byte of it
 *   that it reads, so no state carries over, but calls whose executions
 *   overlap on the GPU (different streams, or different host threads) race
 *   on the array and produce wrong results: serialise them. */
#define GB_STATIC_SCRATCH_BYTES (32u << 20)
GB_API int gb_sgemm_noalloc(gb_handle_t h, gb_algo_t algo, char transa, char transb,
                            int64_t m, int64_t n, int64_t k,
                            float alpha, const float *A, int64_t lda,
                            const float *B, int64_t ldb,
                            float beta, float *C, int64_t ldc, void *stream);

/* Pack-once, multiply-many interface of the split algorithms (the paper
 * re-buffers B' into a contiguous block before the inner loop, Sec. 3;
 * here a whole operand is split and re-laid out once and can then be reused
 * across calls, e.g. a weight matrix).
 *
 * gb_sgemm_pack_size: bytes of one packed operand. which = 'A' packs op(A)
 * (mn = M rows, K columns); which = 'B' packs op(B) (mn = N columns, K rows).
 * Layout (opaque to callers): terms x mn x kpad elements, K contiguous.
 * gb_sgemm_pack: split and pack op(X) of stored matrix X (trans, ldx as in
 * gb_sgemm: X is mn x K if trans is 'N' and which is 'A', and so on) into
 * `packed` (256-byte aligned, >= gb_sgemm_pack_size bytes).
 * gb_sgemm_compute: C <- alpha*op(A)*op(B) + beta*C from packed operands made
 * with the same algorithm and K. Together, pack A + pack B + compute do
 * what gb_sgemm does for a split algorithm, bit for bit, except that
 * gb_sgemm may also split K across CTAs (few output tiles, K >= 1024; the
 * partial sums then go through its workspace), which compute never does.
 * algo must be a split algorithm or AUTO resolved by K to one
 * (GB_ERR_UNSUPPORTED for SIMT). Negative codes: -1 which/trans invalid
 * (pack), -3 mn or M < 0, -4 N < 0, -5 K < 0, -8 ldx too small, -13 ldc. */
GB_API int gb_sgemm_pack_size(gb_algo_t algo, char which, int64_t mn, int64_t k, size_t *bytes);
GB_API int gb_sgemm_pack(gb_handle_t h, gb_algo_t algo, char which, char trans, int64_t mn,
                         int64_t k, const float *X, int64_t ldx, void *packed, size_t bytes,
                         void *stream);
GB_API int gb_sgemm_compute(gb_handle_t h, gb_algo_t algo, int64_t m, int64_t n, int64_t k,
                            float alpha, const void *Apacked, const void *Bpacked, float beta,
                            float *C, int64_t ldc, void *stream);

/* Gradients of C = alpha*op(A)*op(B) + beta*C_in with respect to A, B and
 * C_in, given dC = dL/dC (M x N, lddc). Any of dA, dB, dCin may be NULL to
 * skip it. dA has the stored shape of A (ldda), dB that of B (lddb), dCin is
 * M x N (lddcin). Each output is overwritten (not accumulated):
 *   op(A) = A   : dA = alpha * dC * op(B)^T
 *   op(A) = A^T : dA = alpha * op(B) * dC^T
 *   op(B) = B   : dB = alpha * op(A)^T * dC
 *   op(B) = B^T : dB = alpha * dC^T * op(A)
 *   dCin = beta * dC
 * Each gradient product runs through gb_sgemm with the same algorithm;
 * `workspace` must hold the larger of the two products' requirements
 * (gb_sgemm_backward_workspace_size). Enqueues on `stream`. */
GB_API int gb_sgemm_backward(gb_handle_t h, gb_algo_t algo, char transa, char transb,
                             int64_t m, int64_t n, int64_t k, float alpha,
                             const float *A, int64_t lda, const float *B, int64_t ldb,
                             float beta, const float *dC, int64_t lddc,
                             float *dA, int64_t ldda, float *dB, int64_t lddb,
                             float *dCin, int64_t lddcin,
                             void *workspace, size_t ws_bytes, void *stream);

/* Workspace bytes for gb_sgemm_backward with the same arguments. */
GB_API int gb_sgemm_backward_workspace_size(gb_algo_t algo, char transa, char transb,
                                            int64_t m, int64_t n, int64_t k,
                                            size_t *bytes);

/* One problem of a grouped call; pointers are device pointers. */
typedef struct {
    char transa, transb;
    int64_t m, n, k;
    float alpha, beta;
    const float *A; int64_t lda;
    const float *B; int64_t ldb;
    float *C; int64_t ldc;
} gb_gemm_problem_t;

/* Plan `count` independent SGEMMs (host array `host_problems`) for one
 * persistent grouped launch. Validates every problem (on error returns
 * -i for the i-th argument of the first bad problem and writes its index to
 * *bad_index if not NULL), sorts the work into tiles, uploads the work list
 * to device memory owned by the plan, and writes the workspace the run needs
 * to *ws_bytes. Synchronises the device; not capturable.
 * Every problem meets the plain FP32 bound 2*max(K,1)*u*D, whatever algo:
 *  GB_ALGO_SIMT  every problem on the CUDA cores;
 *  GB_ALGO_AUTO  per problem: an autotuner (run once per handle, timing
 *                synthetic groups) routes each size class to SIMT or the
 *                tensor cores; tensor-core problems take SPLIT_BF16X3 when
 *                K >= 1024 (if those fill at least one round of the
 *                persistent grid, else they join the next), else
 *                SPLIT_BF16X6;
 *  a split algo  the preferred split for every problem with K >= 9; a
 *                problem whose K is below that split's threshold (see
 *                gb_algo_t) takes SPLIT_BF16X6 instead.
 * Problems with K < 9, alpha = 0 or K = 0 always run on the CUDA cores.
 * The tensor-core problems of one split run in one persistent launch. */
GB_API int gb_sgemm_grouped_plan(gb_handle_t h, gb_algo_t algo, int64_t count,
                                 const gb_gemm_problem_t *host_problems,
                                 gb_grouped_plan_t *plan, size_t *ws_bytes,
                                 int64_t *bad_index);

/* Run a plan: enqueues a fixed sequence of kernels on `stream`, with no
 * allocation and no host synchronisation, so it may be captured in a CUDA
 * graph. `workspace` must be 256-byte aligned and at least the planned size. */
GB_API int gb_sgemm_grouped_run(gb_grouped_plan_t plan, void *workspace, size_t ws_bytes,
                                void *stream);

/* Free a plan's device memory (synchronises the device). NULL is a no-op. */
GB_API int gb_sgemm_grouped_destroy(gb_grouped_plan_t plan);

/* Error report of an FP32 result C (M x N) against an FP64 reference C64
 * and bound denominator D (both M x N, column-major, device pointers):
 *   ratio_ij = |C_ij - C64_ij| / (2 * max(K,1) * 2^-24 * D_ij)
 * with ratio 0 where numerator and bound are both 0 and +inf where only the
 * bound is 0; two NaNs or equal infinities agree (ratio 0), one non-finite
 * side alone gives +inf. Reports the maximum ratio, the lower median (rank
 * floor((MN-1)/2) in ascending order, found exactly by radix selection on the
 * FP64 bit patterns), sum |C - C64|^2, sum C64^2 (finite entries), the
 * count of ratios > 1 and the number of elements. This is the only FP64
 * arithmetic on the GPU. Synchronises `stream` and writes *out.
 * `workspace` needs gb_err_report_workspace_size(m, n) bytes. */
typedef struct {
    double max_ratio;
    double median_ratio;
    double sum_sq_diff;
    double sum_sq_ref;
    int64_t n_fail;
    int64_t count;
} gb_err_report_t;

GB_API size_t gb_err_report_workspace_size(int64_t m, int64_t n);
GB_API int gb_err_report(gb_handle_t h, int64_t m, int64_t n, int64_t k,
                         const float *C, int64_t ldc, const double *C64, int64_t ldc64,
                         const double *D, int64_t ldd, void *workspace, size_t ws_bytes,
                         gb_err_report_t *out, void *stream);

/* Synchronise `stream`, then read and clear the handle's device error word.
 * Returns GB_OK if no bounded wait expired since the last call, else
 * GB_ERR_TIMEOUT and writes the id of the wait site to *site (if not NULL). */
GB_API int gb_get_device_error(gb_handle_t h, void *stream, int *site);

/* Time limit of each bounded mbarrier wait in the tensor-core kernels, in
 * microseconds of GPU wall clock (default 2,000,000 = 2 s). A wait that
 * runs out records its site in the device error word and the kernel leaves
 * cleanly (see gb_get_device_error). Values < 1 are rejected (GB_ERR_ARG). */
GB_API int gb_set_wait_limit(gb_handle_t h, int64_t microseconds);

/* Whether gb_sgemm (and gb_sgemm_backward) may split the operands inside the
 * tensor-core kernel instead of in a separate split/pack pass (default: 0).
 * The fused form applies to SPLIT_BF16X3 and SPLIT_BF16X6 when A and B are
 * 16-byte aligned with leading dimensions that are multiples of 4; it reads
 * the FP32 operands once and needs no operand workspace (the workspace is
 * still required for split-K partials). It consumes K in 32-element stages,
 * so for K > 2048 its results are bit-identical to the two-pass form's. It
 * is off by default because it measured slower than the two-pass form: its in-place
 * conversion moves each operand stage through shared memory three times
 * (9.2 ms against 1.9 ms at M = N = K = 8192). */
GB_API int gb_set_fused_split(gb_handle_t h, int enable);

/* Whether gb_sgemm (and the calls built on it) may take the skinny-product
 * kernel (default: 1). It applies to SPLIT_BF16X3, SPLIT_BF16X6 and SPLIT_BF16X9 (and AUTO
 * when it resolves to one of them) when one side has at most 64 rows
 * (M <= 64 or N <= 64), K >= 256, the long side times K is at least 2^22,
 * promotion is off, and TMA can read the long operand in place (16-byte
 * aligned, leading dimension a multiple of 4). Such a product is bound by
 * reading the long operand once: the kernel reads it as FP32 and splits it
 * in shared memory on its way to the tensor cores (paper Sec. 3, the
 * re-buffering of B'), packs only the short operand, and spreads the
 * k-blocks evenly over the SMs (stream-K); a tile shared by several SMs is
 * summed by the last of them in a fixed order, so results are deterministic.
 * The workspace of gb_sgemm_workspace_size covers it. Off: the two-pass
 * form (split/pack pass, then the tensor-core kernel) runs instead.
 * gb_get_skinny_split reads the setting back (GB_ERR_ARG for a null
 * pointer). */
GB_API int gb_set_skinny_split(gb_handle_t h, int enable);
GB_API int gb_get_skinny_split(gb_handle_t h, int *enable);

/* Promoted accumulation in the split algorithms' tensor-core kernel
 * (default 0 = off). The tensor cores add the term products of a tile into
 * an FP32 accumulator in tensor memory, and that addition is not IEEE
 * round-to-nearest: it truncates, so its errors share a sign and grow with
 * the number of accumulation steps. With k_chunk > 0 the kernel starts a
 * fresh accumulator for every k_chunk elements of K (rounded up to whole
 * k-blocks of 32 elements for the BF16 splits, 16 for TF32X3) and adds the
 * finished chunks on the CUDA cores in FP32 with round-to-nearest, in K
 * order, into a running sum kept in registers; the α/β epilogue then reads
 * that sum. The truncation then acts only within a chunk. The product is
 * the same (paper Sec. 1); only the order and rounding of the additions
 * change, so every algorithm keeps its error bound, and the measured error
 * falls (see the accuracy report of the benchmark). With k_chunk >= K the
 * result equals the unpromoted kernel's with 64-byte rows bit for bit.
 * Applies to gb_sgemm, gb_sgemm_compute, gb_sgemm_backward, gb_sgemm_host
 * and the GEMMs inside gb_strsm and the training step (which then apply
 * their elementwise operations in separate passes); grouped runs, gb_ssyrk
 * and the fused in-kernel split (gb_set_fused_split) do not promote.
 * GB_ERR_ARG for k_chunk < 0. gb_get_promotion reads the setting back. */
GB_API int gb_set_promotion(gb_handle_t h, int64_t k_chunk);
GB_API int gb_get_promotion(gb_handle_t h, int64_t *k_chunk);

/* ---------------------------------------------------------------------
 * Autotuning and its cache (the paper chose its block sizes
 * experimentally, Sec. 3; here the library measures its own choices).
 *
 * gb_tune_grouped runs the grouped autotuner now: for each size class of a
 * problem (floor(log2) of the geometric mean of M, N, K, 8 classes from 8
 * to 1024) it times synthetic groups under SIMT with 64 x 64 tiles, SIMT
 * with 128 x 128 tiles, and the tensor cores in each grouped kernel
 * configuration (0: 128 x 128 tiles, 64-byte rows, two CTAs per SM; 1:
 * 128 x 256 tiles, 64-byte rows, one CTA per SM; 2: 128 x 128 tiles,
 * 128-byte rows, one CTA per SM; the stage count follows from each), keeps
 * the fastest per class, then checks the result on one mixed group. AUTO
 * plans run it on first use if the handle has no result yet; split-algorithm
 * plans use its configurations when present. Synchronises; allocates and
 * frees scratch memory.
 *
 * gb_tune_sgemm times gb_sgemm's tensor-core kernel for this algorithm and
 * shape with 64-byte and with 128-byte shared-memory rows (scratch inputs of
 * that shape) and records the faster for the shape's bucket (the split mode
 * and floor(log2) of M, N and K); later gb_sgemm calls of that bucket use it
 * instead of the built-in rule (the environment variable
 * GB_SGEMM_TC_ROW_BYTES still overrides both). Synchronises; allocates and
 * frees scratch memory. GB_ERR_UNSUPPORTED for SIMT or when the table is
 * full.
 *
 * The results form a gb_tuning_t, keyed by the GPU's name, its SM count,
 * the CUDA runtime version and the library version. gb_tuning_write and
 * gb_tuning_read store and load one as a small JSON file (host only, no
 * device needed; GB_ERR_ARG for a file that is missing or malformed).
 * gb_get_tuning / gb_set_tuning copy a record out of or into a handle;
 * gb_set_tuning returns GB_ERR_ARG when the record's key does not match the
 * handle's device. When the environment variable GB_SGEMM_TUNING names a
 * file, gb_create loads it if its key matches, and every tuning call that
 * changes the handle's record writes it back there.
 * ------------------------------------------------------------------- */
#define GB_TUNING_MAX_GEMM 64
typedef struct {
    int mode;                  /* split mode: 0 TF32X3, 1 BF16X3, 2 BF16X6, 3 BF16X9, 4 FP16X3 */
    int log2_m, log2_n, log2_k;
    int row_bytes;             /* 64 or 128 */
} gb_tuning_gemm_t;
typedef struct {
    char gpu_name[96];
    int sm_count;
    int cuda_runtime_version;
    int library_version;
    int grouped_valid;         /* 1 when grouped_route holds a tuned result */
    int grouped_route[8];      /* per size class: 0 SIMT 64x64, 1 SIMT 128x128, 2 + v tensor cores, configuration v */
    int n_gemm;                /* entries of gemm[] in use */
    gb_tuning_gemm_t gemm[GB_TUNING_MAX_GEMM];
} gb_tuning_t;

GB_API int gb_tune_grouped(gb_handle_t h);
GB_API int gb_tune_sgemm(gb_handle_t h, gb_algo_t algo, char transa, char transb, int64_t m,
                         int64_t n, int64_t k);
GB_API int gb_get_tuning(gb_handle_t h, gb_tuning_t *t);
GB_API int gb_set_tuning(gb_handle_t h, const gb_tuning_t *t);
GB_API int gb_tuning_write(const gb_tuning_t *t, const char *path);
GB_API int gb_tuning_read(gb_tuning_t *t, const char *path);

/* Device workspace bytes gb_sgemm_host needs for this problem. */
GB_API int gb_sgemm_host_workspace_size(gb_algo_t algo, char transa, char transb, int64_t m,
                                        int64_t n, int64_t k, size_t *bytes);

/* gb_sgemm with A, B and C in HOST memory (page-locked memory lets the
 * copies overlap; pageable memory works, slower). Arguments, semantics and
 * status codes as gb_sgemm; `workspace` is DEVICE memory (256-byte aligned)
 * of at least gb_sgemm_host_workspace_size bytes. op(A) is copied once (and
 * split and packed once for a split algorithm); op(B) and C then move in
 * blocks of columns through two device slots, so that the host->device copy
 * of block j+1, the GEMM of block j and the device->host copy of block j-1
 * run concurrently on three streams owned by the handle. The pipeline starts
 * after the work already enqueued on `stream`, and `stream` waits for its
 * last copy: the call is ordered on `stream` and returns without waiting
 * (the host buffers must stay valid until `stream` has reached that point).
 * Calls on one handle must not run concurrently from several host threads.
 * For a split algorithm the per-block GEMMs use no split-K, so results can
 * differ in rounding from gb_sgemm's on shapes where gb_sgemm splits K. */
GB_API int gb_sgemm_host(gb_handle_t h, gb_algo_t algo, char transa, char transb, int64_t m,
                         int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
                         const float *B, int64_t ldb, float beta, float *C, int64_t ldc,
                         void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------
 * Training step of a fully connected network on the SGEMM (the paper's
 * application, Sec. 4: the SGEMM as the kernel of neural-network training).
 *
 * Layers l = 1..L with widths n_0..n_L; examples are columns. All matrices
 * are column-major FP32 device arrays with leading dimension = rows:
 *   X  n_0 x B (input),  Y  n_L x B (target),
 *   W[l-1]  n_l x n_{l-1},  b[l-1]  n_l,  H[l-1], G[l-1]  n_l x B.
 * W, b, H and G are HOST arrays of L device pointers. The network:
 *   H_l = phi_l(W_l H_{l-1} + b_l 1^T),  H_0 = X,
 *   phi_l = `hidden` for l < L, identity for l = L;
 *   loss E = sum_ij (H_L - Y)_ij^2 / (2B).
 * No two of these buffers may overlap.
 * Every GEMM runs through gb_sgemm with `algo` (its error bound applies per
 * GEMM); the elementwise passes and the fixed-order reductions run in the
 * library's own kernels. On an error nothing more is enqueued; work already
 * enqueued is not undone. The calls are asynchronous on `stream`; the
 * workspace must be 256-byte aligned and at least gb_mlp_workspace_size.
 * ------------------------------------------------------------------- */
typedef enum { GB_ACT_IDENTITY = 0, GB_ACT_TANH = 1 } gb_activation_t;

typedef struct {
    int64_t layers;            /* L >= 1 */
    const int64_t *widths;     /* host array n_0 .. n_L, each >= 1 */
    int64_t batch;             /* B >= 1 */
    gb_activation_t hidden;    /* activation of layers 1 .. L-1 */
} gb_mlp_desc_t;

/* Workspace bytes of gb_mlp_forward (train = 0) or gb_mlp_train_step
 * (train != 0). GB_ERR_ARG for an invalid description or algo. */
GB_API int gb_mlp_workspace_size(gb_algo_t algo, const gb_mlp_desc_t *desc, int train,
                                 size_t *bytes);

/* Forward pass: writes H_1 .. H_L. */
GB_API int gb_mlp_forward(gb_handle_t h, gb_algo_t algo, const gb_mlp_desc_t *desc,
                          const float *const *W, const float *const *b, const float *X,
                          float *const *H, void *workspace, size_t ws_bytes, void *stream);

/* One step of gradient descent with learning rate lr: the forward pass
 * (H_1 .. H_L), the loss E into *loss (one float, device), the backward
 * pass G_l = dE/dZ_l with Z_l = W_l H_{l-1} + b_l 1^T:
 *   G_L = (H_L - Y) / B,  G_l = (W_{l+1}^T G_{l+1}) * phi'(Z_l)
 * (tanh' = 1 - H_l^2, formed with the weights before the update), and the
 * update W_l <- W_l - lr G_l H_{l-1}^T (one SGEMM with alpha = -lr and
 * beta = 1 on W_l), b_l <- b_l - lr G_l 1 (row sums in a fixed order). */
GB_API int gb_mlp_train_step(gb_handle_t h, gb_algo_t algo, const gb_mlp_desc_t *desc,
                             float *const *W, float *const *b, const float *X, const float *Y,
                             float lr, float *const *H, float *const *G, float *loss,
                             void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------
 * SSYRK and STRSM on the SGEMM core (Level-3 BLAS, whose routines are
 * written over GEMM; the paper's SGEMM implements the Level-3 BLAS SGEMM
 * interface, Sec. 1). Asynchronous on `stream`; the workspace (256-byte
 * aligned) must hold gb_*_workspace_size bytes (0 means none is needed).
 * ------------------------------------------------------------------- */

/* Workspace bytes of gb_ssyrk with these arguments. */
GB_API int gb_ssyrk_workspace_size(gb_algo_t algo, char uplo, char trans, int64_t n, int64_t k,
                                   size_t *bytes);

/* C <- alpha*op(A)*op(A)^T + beta*C on the `uplo` ('U' or 'L') triangle of
 * the n x n matrix C; the other triangle is neither read nor written.
 * op(A) = A (n x k, lda >= max(1, n)) for trans 'N', A^T (A k x n,
 * lda >= max(1, k)) for 'T' or 'C'; ldc >= max(1, n). C is not read when
 * beta = 0; A is not read when alpha = 0 or k = 0. Negative returns are
 * BLAS argument positions (1 uplo, 2 trans, 3 n, 4 k, 7 lda, 10 ldc).
 * With a split algorithm (AUTO: K >= 9) op(A) is split and packed once into
 * the workspace and the whole triangle runs in one tensor-core launch (the
 * algorithm's error bound per element, as for gb_sgemm). With SIMT, or when
 * alpha = 0 or K = 0, it recurses by halving: each level's off-diagonal
 * block is one gb_sgemm call and the diagonal blocks (at most 128 rows) run
 * in FP32 on the CUDA cores. */
GB_API int gb_ssyrk(gb_handle_t h, gb_algo_t algo, char uplo, char trans, int64_t n, int64_t k,
                    float alpha, const float *A, int64_t lda, float beta, float *C, int64_t ldc,
                    void *workspace, size_t ws_bytes, void *stream);

/* Workspace bytes of gb_strsm with these arguments: the GEMM updates' need
 * (256-byte rounded) plus 140,288 bytes per 256 rows of A's diagonal, where
 * each diagonal block's triangle and diagonal reciprocals are laid out once
 * per call for the substitution kernels; for AUTO and the BF16 splits also
 * op(A) and X in split form (three BF16 terms each: 6 * s * kpad bytes for
 * op(A) and 6 * v * kpad for X, s = m (side 'L') or n, v the other
 * dimension, kpad = s rounded up to a multiple of 8). */
GB_API int gb_strsm_workspace_size(gb_algo_t algo, char side, char uplo, char transa, char diag,
                                   int64_t m, int64_t n, size_t *bytes);

/* Solves op(A) X = alpha B (side 'L', A m x m) or X op(A) = alpha B (side
 * 'R', A n x n) for X (m x n), which overwrites B. A is triangular: only
 * its `uplo` triangle is read, and with diag 'U' its diagonal is taken as 1
 * and not read. lda >= max(1, m or n), ldb >= max(1, m). B is scaled by
 * alpha first; alpha = 0 sets B to 0 without reading A or B. A singular A
 * gives infinities or NaNs, as in BLAS. Negative returns are BLAS argument
 * positions (1 side, 2 uplo, 3 transa, 4 diag, 5 m, 6 n, 9 lda, 11 ldb).
 * Recursion by halving: each level's off-diagonal block update is a GEMM
 * with `algo` (alpha = -1, beta = 1), and the diagonal blocks (at most 256
 * rows) are solved by substitution in FP32, with each diagonal entry's
 * reciprocal rounded once. For AUTO and the BF16 splits, op(A) is split
 * once per call and the substitution kernels also write X in split form, so
 * each update is one tensor-core launch on views of the two (the same
 * terms and products as a gb_sgemm of the blocks); for the other
 * algorithms each update is one gb_sgemm call. The handle keeps the last
 * call's launches as an instantiated CUDA graph: a call with the same
 * arguments (pointers included) and handle settings replays it, any other
 * call captures anew (on a stream of the handle; the first call of a given
 * set of arguments therefore costs the capture too). Inside the caller's
 * own stream capture the launches go straight into that capture. The
 * cache makes a handle unsafe for gb_strsm calls from several host threads
 * at once. `workspace` (16-byte aligned, at least
 * gb_strsm_workspace_size bytes) is always needed when m, n > 0 and alpha != 0;
 * otherwise GB_ERR_WORKSPACE. */
GB_API int gb_strsm(gb_handle_t h, gb_algo_t algo, char side, char uplo, char transa, char diag,
                    int64_t m, int64_t n, float alpha, const float *A, int64_t lda, float *B,
                    int64_t ldb, void *workspace, size_t ws_bytes, void *stream);

/* Measurement aid (the paper has no counterpart): enqueues one launch of
 * an FP32 FMA throughput kernel (8 blocks of 256 threads per SM, 128
 * independent fused multiply-adds per thread per iteration) on `stream` and
 * writes the number of FMAs it performs to *fmas. The caller times it (CUDA
 * events) to measure the FP32 SIMT roofline: 2 * fmas / time. `sink` is a
 * device buffer of at least 256 floats (written only to keep the work
 * live). */
GB_API int gb_measure_ffma(gb_handle_t h, int64_t iterations, float *sink, int64_t *fmas,
                           void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSGEMM_H */
