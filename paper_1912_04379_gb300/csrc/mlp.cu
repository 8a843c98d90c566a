// One training step of a fully connected network with the SGEMM as its kernel
// (the paper's application: distributed training of a large neural network,
// Sec. 4). Examples are columns: X is n_0 x B, layer l has weights W_l
// (n_l x n_{l-1}, column-major, ld = n_l), bias b_l and output H_l (n_l x B).
//
//   forward   H_l = phi_l(W_l H_{l-1} + b_l 1^T)        sgemm, bias + act in its epilogue
//   loss      E = sum (H_L - Y)^2 / (2B),  G_L = (H_L - Y) / B
//   backward  G_{l-1} = (W_l^T G_l) * phi'(H_{l-1})     sgemm, * (1 - H^2) in its epilogue
//             W_l <- W_l - lr G_l H_{l-1}^T               one sgemm, alpha = -lr, beta = 1
//             b_l <- b_l - lr G_l 1                       bias_partial + bias_apply
//
// The weight update is the gradient GEMM itself (beta = 1 on W_l), so no
// gradient matrix is stored. G_{l-1} is formed before W_l is overwritten.
// The bias/activation and the tanh' factor run in the tensor-core GEMM's
// epilogue when the algorithm resolves to BF16 x 2 or x 3 terms without
// split-K (rounding exactly as the separate passes); otherwise bias_act and
// tanh_grad run as passes of their own.
// Every elementwise pass is a grid-stride, HBM-bound kernel; every reduction
// (loss, bias) sums in a fixed order, so a step is deterministic on a device.
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace gb {
namespace {

constexpr int kThreads = 256;
constexpr int kBiasChunks = 64;        // column chunks of the bias row sums
constexpr int kLossBlocksMax = 1024;

// H <- act(H + b 1^T) over an n x B column-major matrix with ld = n. The
// row index follows the flat grid-stride index incrementally (no division
// inside the loop).
__global__ void __launch_bounds__(kThreads)
bias_act_kernel(int64_t n, int64_t total, float *__restrict__ H, const float *__restrict__ b,
                int tanh_act) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t step_i = stride % n;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = idx % n;
    for (; idx < total; idx += stride) {
        const float v = H[idx] + b[i];
        H[idx] = tanh_act ? tanhf(v) : v;
        i += step_i;
        if (i >= n) i -= n;
    }
}

// G <- (H - Y) / B, and per-block partial sums of (H - Y)^2 (fixed order:
// each thread its grid-stride elements in order, then a fixed tree).
__global__ void __launch_bounds__(kThreads)
loss_grad_kernel(int64_t total, float fb, const float *__restrict__ H, const float *__restrict__ Y,
                 float *__restrict__ G, float *__restrict__ partial) {
    __shared__ float red[kThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const float d = H[idx] - Y[idx];
        G[idx] = d / fb;
        acc = fmaf(d, d, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

// loss = (sum of the partials) / (2B), one block of kThreads threads: thread
// t sums partials t, t + kThreads, ... in order, then a fixed tree.
__global__ void __launch_bounds__(kThreads)
loss_finish_kernel(const float *__restrict__ partial, int nblocks, float fb,
                   float *__restrict__ loss) {
    __shared__ float red[kThreads / 32];
    float s = 0.f;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) s += partial[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        *loss = t / (2.f * fb);
    }
}

// G <- G * (1 - H^2): tanh'(Z) written through H = tanh(Z).
__global__ void __launch_bounds__(kThreads)
tanh_grad_kernel(int64_t total, float *__restrict__ G, const float *__restrict__ H) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const float h = H[idx];
        G[idx] = G[idx] * fmaf(-h, h, 1.f);
    }
}

// partial[c * n + i] = sum over columns j of chunk c of G[i + j n] (in order).
__global__ void __launch_bounds__(kThreads)
bias_partial_kernel(int64_t n, int64_t B, int64_t cols_per_chunk, const float *__restrict__ G,
                    float *__restrict__ partial) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j0 = (int64_t)blockIdx.y * cols_per_chunk;
    const int64_t j1 = j0 + cols_per_chunk < B ? j0 + cols_per_chunk : B;
    float s = 0.f;
    for (int64_t j = j0; j < j1; ++j) s += G[i + j * n];
    partial[(int64_t)blockIdx.y * n + i] = s;
}

// b_i <- b_i - lr * (sum of the chunk partials, in order)
__global__ void __launch_bounds__(kThreads)
bias_apply_kernel(int64_t n, int nchunks, const float *__restrict__ partial, float lr,
                  float *__restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)c * n + i];
    b[i] = fmaf(-lr, s, b[i]);
}

int grid_for(int64_t total, int sm_count) {
    const int64_t want = (total + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 1) * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Plan {
    size_t gemm_ws = 0, bias_off = 0, loss_off = 0, total = 0;
};

// Validates a description; fills the workspace layout for `train` (which also
// needs the backward GEMMs and the reductions) or the forward alone.
int layout(gb_algo_t algo, const gb_mlp_desc_t *d, bool train, Plan *p) {
    if (!d || !d->widths || d->layers < 1 || d->layers > 4096 || d->batch < 1) return GB_ERR_ARG;
    if (d->hidden != GB_ACT_IDENTITY && d->hidden != GB_ACT_TANH) return GB_ERR_ARG;
    if (algo < GB_ALGO_AUTO || algo > GB_ALGO_SPLIT_FP16X3) return GB_ERR_ARG;
    const int64_t B = d->batch;
    int64_t max_n = 1;
    size_t ws = 0;
    for (int64_t l = 0; l <= d->layers; ++l) {
        if (d->widths[l] < 1 || d->widths[l] > ((int64_t)1 << 31)) return GB_ERR_ARG;
        if ((double)d->widths[l] * (double)B > 70368744177664.0) return GB_ERR_ARG;   // 2^46
    }
    for (int64_t l = 0; l < d->layers; ++l) {
        const int64_t m = d->widths[l + 1], k = d->widths[l];
        if (m > max_n) max_n = m;
        size_t w = 0;
        int rc = gb_sgemm_workspace_size(algo, 'N', 'N', m, B, k, &w);       // forward
        if (rc) return GB_ERR_ARG;
        if (w > ws) ws = w;
        if (!train) continue;
        rc = gb_sgemm_workspace_size(algo, 'N', 'T', m, k, B, &w);           // update
        if (rc) return GB_ERR_ARG;
        if (w > ws) ws = w;
        if (l > 0) {
            rc = gb_sgemm_workspace_size(algo, 'T', 'N', k, B, m, &w);       // G_{l-1}
            if (rc) return GB_ERR_ARG;
            if (w > ws) ws = w;
        }
    }
    p->gemm_ws = round_up(ws, 256);
    p->bias_off = p->gemm_ws;
    const size_t bias_bytes = train ? round_up((size_t)kBiasChunks * (size_t)max_n * 4, 256) : 0;
    p->loss_off = p->bias_off + bias_bytes;
    p->total = p->loss_off + (train ? (size_t)kLossBlocksMax * 4 : 0);
    return GB_OK;
}

int check_handle(gb_handle_t h) {
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    return dev == h->device ? GB_OK : GB_ERR_HANDLE;
}

int check_ptrs(const gb_mlp_desc_t *d, const void *const *xs) {
    if (!xs) return GB_ERR_ARG;
    for (int64_t l = 0; l < d->layers; ++l)
        if (!xs[l]) return GB_ERR_ARG;
    return GB_OK;
}

int forward(gb_handle_t h, gb_algo_t algo, const gb_mlp_desc_t *d, const float *const *W,
            const float *const *b, const float *X, float *const *H, void *ws, size_t ws_bytes,
            cudaStream_t s) {
    const int64_t B = d->batch, L = d->layers;
    for (int64_t l = 0; l < L; ++l) {
        const int64_t m = d->widths[l + 1], k = d->widths[l];
        const float *prev = l ? H[l - 1] : X;
        const int tanh_act = (l < L - 1 && d->hidden == GB_ACT_TANH) ? 1 : 0;
        // bias and activation in the GEMM's epilogue where the tensor-core
        // kernel can take them, else a separate pass
        EpiOp op;
        op.kind = 1;
        op.tanh_act = tanh_act;
        op.bias = b[l];
        bool fused = false;
        int rc = sgemm_epi(h, algo, 'N', 'N', m, B, k, 1.f, W[l], m, prev, k, 0.f, H[l], m, op, ws,
                           ws_bytes, s, &fused);
        if (rc) return rc;
        if (fused) continue;
        const int64_t total = m * B;
        bias_act_kernel<<<grid_for(total, h->sm_count), kThreads, 0, s>>>(m, total, H[l], b[l],
                                                                          tanh_act);
        if (cudaGetLastError() != cudaSuccess) return GB_ERR_CUDA;
    }
    return GB_OK;
}

}  // namespace
}  // namespace gb

extern "C" {

GB_API int gb_mlp_workspace_size(gb_algo_t algo, const gb_mlp_desc_t *desc, int train,
                                 size_t *bytes) {
    if (!bytes) return GB_ERR_ARG;
    gb::Plan p;
    int rc = gb::layout(algo, desc, train != 0, &p);
    if (rc) return rc;
    *bytes = p.total;
    return GB_OK;
}

GB_API int gb_mlp_forward(gb_handle_t h, gb_algo_t algo, const gb_mlp_desc_t *desc,
                          const float *const *W, const float *const *b, const float *X,
                          float *const *H, void *workspace, size_t ws_bytes, void *stream) {
    using namespace gb;
    int rc = check_handle(h);
    if (rc) return rc;
    Plan p;
    rc = layout(algo, desc, false, &p);
    if (rc) return rc;
    if (check_ptrs(desc, (const void *const *)W) || check_ptrs(desc, (const void *const *)b) ||
        check_ptrs(desc, (const void *const *)H) || !X)
        return GB_ERR_ARG;
    if (ws_bytes < p.total || (p.total && (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))))
        return GB_ERR_WORKSPACE;
    return forward(h, algo, desc, W, b, X, H, workspace, p.gemm_ws, static_cast<cudaStream_t>(stream));
}

GB_API int gb_mlp_train_step(gb_handle_t h, gb_algo_t algo, const gb_mlp_desc_t *desc,
                             float *const *W, float *const *b, const float *X, const float *Y,
                             float lr, float *const *H, float *const *G, float *loss,
                             void *workspace, size_t ws_bytes, void *stream) {
    using namespace gb;
    int rc = check_handle(h);
    if (rc) return rc;
    Plan p;
    rc = layout(algo, desc, true, &p);
    if (rc) return rc;
    if (check_ptrs(desc, (const void *const *)W) || check_ptrs(desc, (const void *const *)b) ||
        check_ptrs(desc, (const void *const *)H) || check_ptrs(desc, (const void *const *)G) ||
        !X || !Y || !loss)
        return GB_ERR_ARG;
    if (ws_bytes < p.total || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return GB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const int64_t B = desc->batch, L = desc->layers;
    const float fb = (float)B;

    rc = forward(h, algo, desc, W, b, X, H, ws, p.gemm_ws, s);
    if (rc) return rc;

    // loss and G_L
    {
        const int64_t nL = desc->widths[L], total = nL * B;
        int nblk = grid_for(total, h->sm_count);
        if (nblk > kLossBlocksMax) nblk = kLossBlocksMax;
        float *partial = reinterpret_cast<float *>(ws + p.loss_off);
        loss_grad_kernel<<<nblk, kThreads, 0, s>>>(total, fb, H[L - 1], Y, G[L - 1], partial);
        loss_finish_kernel<<<1, kThreads, 0, s>>>(partial, nblk, fb, loss);
        if (cudaGetLastError() != cudaSuccess) return GB_ERR_CUDA;
    }

    for (int64_t l = L - 1; l >= 0; --l) {
        const int64_t m = desc->widths[l + 1], k = desc->widths[l];
        const float *prev = l ? H[l - 1] : X;
        if (l > 0) {
            // G_{l-1} = W_l^T G_l (with the weights before this step's update),
            // times tanh' = 1 - H_{l-1}^2 in the epilogue where possible
            EpiOp op;
            op.kind = desc->hidden == GB_ACT_TANH ? 2 : 0;
            op.aux = H[l - 1];
            op.ldaux = k;
            bool fused = false;
            rc = sgemm_epi(h, algo, 'T', 'N', k, B, m, 1.f, W[l], m, G[l], m, 0.f, G[l - 1], k, op,
                           ws, p.gemm_ws, s, &fused);
            if (rc) return rc;
            if (desc->hidden == GB_ACT_TANH && !fused) {
                const int64_t total = k * B;
                tanh_grad_kernel<<<grid_for(total, h->sm_count), kThreads, 0, s>>>(total, G[l - 1],
                                                                                  H[l - 1]);
                if (cudaGetLastError() != cudaSuccess) return GB_ERR_CUDA;
            }
        }
        // W_l <- W_l - lr G_l prev^T
        rc = gb_sgemm(h, algo, 'N', 'T', m, k, B, -lr, G[l], m, prev, k, 1.f, W[l], m, ws,
                      p.gemm_ws, s);
        if (rc) return rc;
        // b_l <- b_l - lr G_l 1
        const int nchunks = (int)(B < kBiasChunks ? B : kBiasChunks);
        const int64_t cpc = (B + nchunks - 1) / nchunks;
        float *partial = reinterpret_cast<float *>(ws + p.bias_off);
        dim3 grid((unsigned)((m + kThreads - 1) / kThreads), (unsigned)nchunks);
        bias_partial_kernel<<<grid, kThreads, 0, s>>>(m, B, cpc, G[l], partial);
        bias_apply_kernel<<<(unsigned)((m + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            m, nchunks, partial, lr, b[l]);
        if (cudaGetLastError() != cudaSuccess) return GB_ERR_CUDA;
    }
    return GB_OK;
}

}  // extern "C"
