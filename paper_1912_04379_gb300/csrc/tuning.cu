// Autotuning records of a handle and their JSON cache (gb_tuning_t in
// include/gbsgemm.h): the grouped autotuner's per-size-class routing, and the
// shared-memory row width (64 or 128 bytes) measured per shape bucket for the
// one-GEMM tensor-core kernel. The JSON reader and writer are plain host code
// and need no device.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "internal.h"

namespace gb {
namespace {

int floor_log2(int64_t x) {
    int l = 0;
    while (x > 1) { x >>= 1; ++l; }
    return l;
}

// ------------------------------------------------------------- JSON I/O --
// The cache is one flat object of known keys: strings, integers, an integer
// array and an array of integer 5-tuples. The reader accepts exactly what the
// writer produces, with any whitespace.

const char *skip_ws(const char *p) {
    while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t') ++p;
    return p;
}

// Position just after `"key":` in the text, or nullptr.
const char *find_key(const std::string &text, const char *key) {
    const std::string pat = std::string("\"") + key + "\"";
    size_t at = text.find(pat);
    if (at == std::string::npos) return nullptr;
    const char *p = skip_ws(text.c_str() + at + pat.size());
    if (*p != ':') return nullptr;
    return skip_ws(p + 1);
}

bool parse_int(const char *&p, int *out) {
    p = skip_ws(p);
    char *end = nullptr;
    const long v = strtol(p, &end, 10);
    if (end == p) return false;
    *out = (int)v;
    p = skip_ws(end);
    return true;
}

bool expect(const char *&p, char c) {
    p = skip_ws(p);
    if (*p != c) return false;
    p = skip_ws(p + 1);
    return true;
}

bool read_int_key(const std::string &text, const char *key, int *out) {
    const char *p = find_key(text, key);
    return p && parse_int(p, out);
}

}  // namespace

// Row width recorded for this call's bucket, 0 if none.
int tuned_row_bytes(gb_handle_t h, int mode, int64_t m, int64_t n, int64_t k) {
    const int lm = floor_log2(m), ln = floor_log2(n), lk = floor_log2(k);
    for (int i = 0; i < h->n_gemm_rb; ++i) {
        const gb_tuning_gemm_t &g = h->gemm_rb[i];
        if (g.mode == mode && g.log2_m == lm && g.log2_n == ln && g.log2_k == lk) return g.row_bytes;
    }
    return 0;
}

// Writes the handle's record to the file named by GB_SGEMM_TUNING, if set.
void tuning_autosave(gb_handle_t h) {
    const char *path = getenv("GB_SGEMM_TUNING");
    if (!path || !*path) return;
    gb_tuning_t t;
    if (gb_get_tuning(h, &t) == GB_OK) gb_tuning_write(&t, path);
}

// Loads the file named by GB_SGEMM_TUNING into a new handle when its key
// matches the handle's device (anything else is ignored).
void tuning_autoload(gb_handle_t h) {
    const char *path = getenv("GB_SGEMM_TUNING");
    if (!path || !*path) return;
    gb_tuning_t t;
    if (gb_tuning_read(&t, path) == GB_OK) gb_set_tuning(h, &t);
}

}  // namespace gb

extern "C" {

GB_API int gb_tuning_write(const gb_tuning_t *t, const char *path) {
    if (!t || !path || t->n_gemm < 0 || t->n_gemm > GB_TUNING_MAX_GEMM) return GB_ERR_ARG;
    // the GPU name goes out with quotes and backslashes removed
    char name[sizeof(t->gpu_name)];
    size_t j = 0;
    for (size_t i = 0; i < sizeof(t->gpu_name) && t->gpu_name[i]; ++i)
        if (t->gpu_name[i] != '"' && t->gpu_name[i] != '\\' && (unsigned char)t->gpu_name[i] >= 32)
            name[j++] = t->gpu_name[i];
    name[j] = 0;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return GB_ERR_ARG;
    fprintf(f, "{\n  \"format\": \"gbsgemm-tuning-1\",\n  \"gpu_name\": \"%s\",\n", name);
    fprintf(f, "  \"sm_count\": %d,\n  \"cuda_runtime_version\": %d,\n  \"library_version\": %d,\n",
            t->sm_count, t->cuda_runtime_version, t->library_version);
    fprintf(f, "  \"grouped_valid\": %d,\n  \"grouped_route\": [", t->grouped_valid);
    for (int c = 0; c < 8; ++c) fprintf(f, "%s%d", c ? ", " : "", t->grouped_route[c]);
    fprintf(f, "],\n  \"gemm\": [");
    for (int i = 0; i < t->n_gemm; ++i) {
        const gb_tuning_gemm_t &g = t->gemm[i];
        fprintf(f, "%s\n    [%d, %d, %d, %d, %d]", i ? "," : "", g.mode, g.log2_m, g.log2_n,
                g.log2_k, g.row_bytes);
    }
    fprintf(f, "%s]\n}\n", t->n_gemm ? "\n  " : "");
    const bool ok = fclose(f) == 0;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return GB_ERR_ARG;
    }
    return GB_OK;
}

GB_API int gb_tuning_read(gb_tuning_t *t, const char *path) {
    using namespace gb;
    if (!t || !path) return GB_ERR_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return GB_ERR_ARG;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 20)) text.append(buf, got);
    fclose(f);
    gb_tuning_t r;
    memset(&r, 0, sizeof(r));
    const char *p = find_key(text, "format");
    if (!p || strncmp(p, "\"gbsgemm-tuning-1\"", 18) != 0) return GB_ERR_ARG;
    p = find_key(text, "gpu_name");
    if (!p || *p != '"') return GB_ERR_ARG;
    ++p;
    size_t j = 0;
    while (*p && *p != '"' && j + 1 < sizeof(r.gpu_name)) r.gpu_name[j++] = *p++;
    if (*p != '"') return GB_ERR_ARG;
    if (!read_int_key(text, "sm_count", &r.sm_count) ||
        !read_int_key(text, "cuda_runtime_version", &r.cuda_runtime_version) ||
        !read_int_key(text, "library_version", &r.library_version) ||
        !read_int_key(text, "grouped_valid", &r.grouped_valid))
        return GB_ERR_ARG;
    p = find_key(text, "grouped_route");
    if (!p || !expect(p, '[')) return GB_ERR_ARG;
    for (int c = 0; c < 8; ++c) {
        if (!parse_int(p, &r.grouped_route[c])) return GB_ERR_ARG;
        if (c < 7 && !expect(p, ',')) return GB_ERR_ARG;
    }
    if (!expect(p, ']')) return GB_ERR_ARG;
    p = find_key(text, "gemm");
    if (!p || !expect(p, '[')) return GB_ERR_ARG;
    while (*p == '[') {
        if (r.n_gemm >= GB_TUNING_MAX_GEMM) return GB_ERR_ARG;
        gb_tuning_gemm_t &g = r.gemm[r.n_gemm++];
        int *v[5] = {&g.mode, &g.log2_m, &g.log2_n, &g.log2_k, &g.row_bytes};
        if (!expect(p, '[')) return GB_ERR_ARG;
        for (int e = 0; e < 5; ++e) {
            if (!parse_int(p, v[e])) return GB_ERR_ARG;
            if (e < 4 && !expect(p, ',')) return GB_ERR_ARG;
        }
        if (!expect(p, ']')) return GB_ERR_ARG;
        if (*p == ',') p = skip_ws(p + 1);
    }
    if (!expect(p, ']')) return GB_ERR_ARG;
    *t = r;
    return GB_OK;
}

GB_API int gb_get_tuning(gb_handle_t h, gb_tuning_t *t) {
    if (!h || h->magic != gb::kHandleMagic) return GB_ERR_HANDLE;
    if (!t) return GB_ERR_ARG;
    memset(t, 0, sizeof(*t));
    memcpy(t->gpu_name, h->gpu_name, sizeof(t->gpu_name));
    t->sm_count = h->sm_count;
    t->cuda_runtime_version = h->cuda_runtime_version;
    t->library_version = gb_version();
    t->grouped_valid = h->grouped_tuned ? 1 : 0;
    for (int c = 0; c < 8; ++c) t->grouped_route[c] = h->grouped_tuned ? h->grouped_choice[c] : 0;
    t->n_gemm = h->n_gemm_rb;
    memcpy(t->gemm, h->gemm_rb, sizeof(t->gemm));
    return GB_OK;
}

GB_API int gb_set_tuning(gb_handle_t h, const gb_tuning_t *t) {
    if (!h || h->magic != gb::kHandleMagic) return GB_ERR_HANDLE;
    if (!t || t->n_gemm < 0 || t->n_gemm > GB_TUNING_MAX_GEMM) return GB_ERR_ARG;
    if (strncmp(t->gpu_name, h->gpu_name, sizeof(t->gpu_name)) != 0 ||
        t->sm_count != h->sm_count || t->cuda_runtime_version != h->cuda_runtime_version ||
        t->library_version != gb_version())
        return GB_ERR_ARG;
    for (int c = 0; c < 8; ++c)
        if (t->grouped_route[c] < 0 || t->grouped_route[c] >= 2 + gb::kGroupedConfigVariants)
            return GB_ERR_ARG;
    for (int i = 0; i < t->n_gemm; ++i) {
        const gb_tuning_gemm_t &g = t->gemm[i];
        if (g.mode < 0 || g.mode > 4 || (g.row_bytes != 64 && g.row_bytes != 128)) return GB_ERR_ARG;
    }
    h->grouped_tuned = t->grouped_valid != 0;
    for (int c = 0; c < 8; ++c) h->grouped_choice[c] = t->grouped_route[c];
    h->n_gemm_rb = t->n_gemm;
    memcpy(h->gemm_rb, t->gemm, sizeof(h->gemm_rb));
    return GB_OK;
}

GB_API int gb_tune_sgemm(gb_handle_t h, gb_algo_t algo, char ta, char tb, int64_t m, int64_t n,
                         int64_t k) {
    using namespace gb;
    if (!h || h->magic != kHandleMagic) return GB_ERR_HANDLE;
    size_t ws_bytes = 0;
    int rc = gb_sgemm_workspace_size(algo, ta, tb, m, n, k, &ws_bytes);
    if (rc) return rc;
    const int mode = split_mode(resolve_algo(algo, k));
    if (mode < 0 || m <= 0 || n <= 0 || k <= 0) return GB_ERR_UNSUPPORTED;
    const int lm = floor_log2(m), ln = floor_log2(n), lk = floor_log2(k);
    int slot = -1;
    for (int i = 0; i < h->n_gemm_rb; ++i) {
        const gb_tuning_gemm_t &g = h->gemm_rb[i];
        if (g.mode == mode && g.log2_m == lm && g.log2_n == ln && g.log2_k == lk) slot = i;
    }
    if (slot < 0 && h->n_gemm_rb >= GB_TUNING_MAX_GEMM) return GB_ERR_UNSUPPORTED;
    const bool tA = ta != 'N' && ta != 'n', tB = tb != 'N' && tb != 'n';
    const int64_t lda = tA ? k : m, ldb = tB ? n : k;
    float *A = nullptr, *B = nullptr, *C = nullptr;
    void *ws = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = GB_ERR_CUDA;
    float best = 1e30f;
    int best_rb = 0;
    if (cudaMalloc(&A, (size_t)m * (size_t)k * 4) == cudaSuccess &&
        cudaMalloc(&B, (size_t)k * (size_t)n * 4) == cudaSuccess &&
        cudaMalloc(&C, (size_t)m * (size_t)n * 4) == cudaSuccess &&
        cudaMalloc(&ws, ws_bytes > 256 ? ws_bytes : 256) == cudaSuccess &&
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMemsetAsync(A, 0x3e, (size_t)m * (size_t)k * 4, s) == cudaSuccess &&
        cudaMemsetAsync(B, 0x3e, (size_t)k * (size_t)n * 4, s) == cudaSuccess) {
        rc = GB_OK;
        const int saved = h->rb_override;
        for (int rb = 64; rb <= 128 && rc == GB_OK; rb *= 2) {
            h->rb_override = rb;
            float t_best = 1e30f;
            for (int rep = 0; rep < 4 && rc == GB_OK; ++rep) {
                cudaEventRecord(e0, s);
                rc = gb_sgemm(h, algo, ta, tb, m, n, k, 1.f, A, lda, B, ldb, 0.f, C, m, ws,
                              ws_bytes > 256 ? ws_bytes : 256, s);
                cudaEventRecord(e1, s);
                if (rc == GB_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = GB_ERR_CUDA;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < t_best) t_best = t;     // the first call warms up
            }
            if (rc == GB_OK && t_best < best) { best = t_best; best_rb = rb; }
        }
        h->rb_override = saved;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(ws);
    cudaFree(C);
    cudaFree(B);
    cudaFree(A);
    if (rc != GB_OK) return rc;
    if (slot < 0) slot = h->n_gemm_rb++;
    h->gemm_rb[slot] = gb_tuning_gemm_t{mode, lm, ln, lk, best_rb};
    tuning_autosave(h);
    return GB_OK;
}

}  // extern "C"
