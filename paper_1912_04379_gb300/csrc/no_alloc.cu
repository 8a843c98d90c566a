// gb_sgemm_noalloc: the split-precision SGEMM for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: a
// plugin running inside a framework that owns every byte of device memory
// through its own pool and forbids raw allocations, code on a latency-
// critical path that cannot afford the implicit device synchronisation an
// allocation may cause, or a process whose device memory is fully reserved
// up front. For them this entry point runs the same kernels as gb_sgemm
// (split/pack of A and B, then the tensor-core kernel), but the split
// workspace lives in one fixed array in device global memory that is part
// of the library itself, so the call allocates nothing.
//
// The array is GB_STATIC_SCRATCH_BYTES (32 MiB) of device memory. Its
// module is loaded on a device, and the array reserved there until the
// process exits, when gb_create looks up the array's device address with
// that device current; the address is kept in the handle. Host code must not
// use the array's name as a device address (on the host it names a stand-in
// object): only the looked-up address is handed to the kernels.
#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_split_scratch[GB_STATIC_SCRATCH_BYTES];

}  // namespace

cudaError_t gb::noalloc_scratch_lookup(void **addr) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_split_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    *addr = p;
    return cudaSuccess;
}

extern "C" GB_API int gb_sgemm_noalloc(gb_handle_t h, gb_algo_t algo, char transa, char transb,
                                       int64_t m, int64_t n, int64_t k, float alpha,
                                       const float *A, int64_t lda, const float *B, int64_t ldb,
                                       float beta, float *C, int64_t ldc, void *stream) {
    size_t need = 0;
    int rc = gb_sgemm_workspace_size(algo, transa, transb, m, n, k, &need);
    if (rc) return rc;
    if (need > (size_t)GB_STATIC_SCRATCH_BYTES) return GB_ERR_WORKSPACE;
    if (!h || h->magic != gb::kHandleMagic) return GB_ERR_HANDLE;
    if (!h->noalloc_scratch) return GB_ERR_CUDA;
    return gb_sgemm(h, algo, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                    h->noalloc_scratch, (size_t)GB_STATIC_SCRATCH_BYTES, stream);
}
