// Planned batches (perm_plan_*), CUDA-graph replay and the chunk-length
// autotuner (perm_tune_*, perm_autotune).
//
// A plan fixes the sizes, the field and (F_p) the primes of a batch: the
// chunk plan is computed, the workspace allocated and the metadata uploaded
// once.  Executing a plan then only enqueues kernels and one memset, so the
// whole pass (staging, one Gray-walk launch per size, finalisation) can be
// captured into a CUDA graph and replayed with a single launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "permx.h"

using namespace permx;

struct perm_plan {
    Prepared X;
    int device = 0;
    int field = 0;
    cudaStream_t capture = nullptr;
    StreamSet streams;               // the size groups' streams (execute and capture)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* gA = nullptr;
    void* gOut = nullptr;
};

// Several plans captured into one CUDA graph: each plan's pass is a branch of
// the graph (and each of its size groups a branch of that), so one launch runs
// every plan's matrices concurrently.
struct perm_graph {
    int device = 0;
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// deterministic fill of synthetic inputs for the autotuner (splitmix64 hash)
__global__ void tune_fill_kernel(unsigned long long* out, int64_t words, uint32_t p, int field) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        if (field == PERMX_FIELD_MODP) {
            reinterpret_cast<uint32_t*>(out)[2 * i] = (uint32_t)(z % p);
            reinterpret_cast<uint32_t*>(out)[2 * i + 1] = (uint32_t)((z >> 32) % p);
        } else {
            reinterpret_cast<double*>(out)[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
        }
    }
}

int check_field(int field) {
    if (field != PERMX_FIELD_C128 && field != PERMX_FIELD_F64 && field != PERMX_FIELD_MODP)
        return fail(PERMX_EINVAL, "unknown field");
    return PERMX_OK;
}

}  // namespace

extern "C" {

int perm_plan_create(int field, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                     void* stream, perm_plan** plan) {
    clear_error();
    if (!plan) return fail(PERMX_EINVAL, "NULL plan pointer");
    int rc = check_field(field);
    if (rc) return rc;
    const int maxn = field == PERMX_FIELD_MODP ? PERMX_MAX_N_MODP : PERMX_MAX_N_FP;
    if (batch < 1) return fail(PERMX_EINVAL, "a plan needs at least one matrix");
    if (!n || !offset) return fail(PERMX_EINVAL, "NULL size or offset array");
    for (int64_t b = 0; b < batch; ++b) {
        if (n[b] < 1 || n[b] > maxn) return fail(PERMX_EINVAL, "n out of range");
        if (offset[b] < 0) return fail(PERMX_EINVAL, "negative offset");
    }
    if (field == PERMX_FIELD_MODP) {
        if (!p) return fail(PERMX_EINVAL, "NULL prime array");
        for (int64_t b = 0; b < batch; ++b)
            if (p[b] <= 2 || p[b] >= (1u << 31) || !is_prime_u32(p[b]))
                return fail(PERMX_EINVAL, "p is not an odd prime below 2^31");
    }
    perm_plan* P = new perm_plan();
    P->field = field;
    cudaGetDevice(&P->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = prepare_batch((Field)field, n, offset, p, batch, s, P->X);
    if (rc) {
        delete P;
        return rc;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = P->streams.create(P->device);
    if (e != cudaSuccess) {
        release_batch(P->X, s);
        if (P->capture) cudaStreamDestroy(P->capture);
        delete P;
        return cuda_fail(e, "perm_plan_create");
    }
    P->X.streams = &P->streams;
    *plan = P;
    return PERMX_OK;
}

int perm_plan_execute(perm_plan* P, const void* A, void* out, void* stream) {
    clear_error();
    if (!P || !A || !out) return fail(PERMX_EINVAL, "NULL argument");
    if (P->field == PERMX_FIELD_C128 && (reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(out) % 16))
        return fail(PERMX_EINVAL, "complex128 arrays must be 16-byte aligned");
    return execute_batch(P->X, A, out, static_cast<cudaStream_t>(stream));
}

int perm_plan_graph_launch(perm_plan* P, const void* A, void* out, void* stream) {
    clear_error();
    if (!P || !A || !out) return fail(PERMX_EINVAL, "NULL argument");
    if (!P->exec || A != P->gA || out != P->gOut) {
        // (re)capture the pass for these buffers on the plan's private stream
        PERMX_CUDA(cudaStreamBeginCapture(P->capture, cudaStreamCaptureModeThreadLocal));
        const int rc = execute_batch(P->X, A, out, P->capture);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(P->capture, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        if (P->exec) cudaGraphExecDestroy(P->exec);
        if (P->graph) cudaGraphDestroy(P->graph);
        P->graph = g;
        P->exec = ex;
        P->gA = A;
        P->gOut = out;
    }
    PERMX_CUDA(cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream)));
    return PERMX_OK;
}

int perm_plan_destroy(perm_plan* P) {
    clear_error();
    if (!P) return fail(PERMX_EINVAL, "NULL plan");
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    release_batch(P->X, P->capture);
    cudaStreamSynchronize(P->capture);
    cudaStreamDestroy(P->capture);
    P->streams.destroy();
    delete P;
    return PERMX_OK;
}

int perm_graph_create(perm_plan* const* plans, const void* const* A, void* const* out, int32_t count,
                      perm_graph** graph) {
    clear_error();
    if (!graph || !plans || !A || !out || count < 1) return fail(PERMX_EINVAL, "bad arguments");
    int dev = 0;
    PERMX_CUDA(cudaGetDevice(&dev));
    for (int32_t i = 0; i < count; ++i) {
        if (!plans[i] || !A[i] || !out[i]) return fail(PERMX_EINVAL, "NULL plan or buffer");
        if (plans[i]->device != dev) return fail(PERMX_EINVAL, "every plan must belong to the current device");
        if (plans[i]->field == PERMX_FIELD_C128 &&
            (reinterpret_cast<uintptr_t>(A[i]) % 16 || reinterpret_cast<uintptr_t>(out[i]) % 16))
            return fail(PERMX_EINVAL, "complex128 arrays must be 16-byte aligned");
        for (int32_t k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(PERMX_EINVAL, "a plan may appear only once in a graph");
    }
    perm_graph* G = new perm_graph();
    G->device = dev;
    cudaError_t e = cudaStreamCreateWithFlags(&G->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (G->capture) cudaStreamDestroy(G->capture);
        delete G;
        return cuda_fail(e, "perm_graph_create");
    }
    int rc = PERMX_OK;
    e = cudaStreamBeginCapture(G->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // fork: every plan's pass starts on that plan's own capture stream
        e = cudaEventRecord(G->fork, G->capture);
        int32_t forked = 0;
        for (; forked < count && e == cudaSuccess; ++forked)
            e = cudaStreamWaitEvent(plans[forked]->capture, G->fork, 0);
        for (int32_t i = 0; i < forked && e == cudaSuccess && rc == PERMX_OK; ++i)
            rc = execute_batch(plans[i]->X, A[i], out[i], plans[i]->capture);
        // join every forked stream back, whatever failed, so the capture can end
        for (int32_t i = 0; i < forked; ++i) {
            cudaError_t f = cudaEventRecord(plans[i]->streams.join[0], plans[i]->capture);
            if (f == cudaSuccess) f = cudaStreamWaitEvent(G->capture, plans[i]->streams.join[0], 0);
            if (e == cudaSuccess) e = f;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(G->capture, &g);
        if (e == cudaSuccess) e = ec;
        if (e == cudaSuccess && rc == PERMX_OK) e = cudaGraphInstantiate(&G->exec, g, 0);
        if (e == cudaSuccess && rc == PERMX_OK) G->graph = g;
        else if (g) cudaGraphDestroy(g);
    }
    if (rc == PERMX_OK && e != cudaSuccess) rc = cuda_fail(e, "perm_graph_create capture");
    if (rc) {
        cudaEventDestroy(G->fork);
        cudaStreamDestroy(G->capture);
        delete G;
        return rc;
    }
    *graph = G;
    return PERMX_OK;
}

int perm_graph_launch(perm_graph* G, void* stream) {
    clear_error();
    if (!G || !G->exec) return fail(PERMX_EINVAL, "NULL graph");
    PERMX_CUDA(cudaGraphLaunch(G->exec, static_cast<cudaStream_t>(stream)));
    return PERMX_OK;
}

int perm_graph_destroy(perm_graph* G) {
    clear_error();
    if (!G) return fail(PERMX_EINVAL, "NULL graph");
    cudaSetDevice(G->device);
    cudaDeviceSynchronize();
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    cudaEventDestroy(G->fork);
    cudaStreamDestroy(G->capture);
    delete G;
    return PERMX_OK;
}

int perm_tune_set(int field, int32_t n, int32_t ell) {
    clear_error();
    int rc = check_field(field);
    if (rc) return rc;
    if (n < 1 || n > PERMX_MAX_N_MODP || ell < 0 || ell > (field == PERMX_FIELD_MODP ? PERMX_MAX_ELL_MODP : PERMX_MAX_ELL_FP))
        return fail(PERMX_EINVAL, "bad n or chunk length");
    tune_set(field, n, ell);
    return PERMX_OK;
}

int perm_tune_get(int field, int32_t n) {
    clear_error();
    int rc = check_field(field);
    if (rc) return rc;
    if (n < 1 || n > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "bad n");
    const int bits = walk_bits(n, 1);
    return chunk_log2((Field)field, n, bits);
}

// Tuning-table persistence.  The file is text: a header line "permx-tune 1",
// then one line "field n ell" per pinned entry.  Saving writes a temporary
// file and renames it over `path`, so a reader never sees half a table;
// loading checks every line against the perm_tune_set limits before it
// changes anything, then replaces the whole table.
int perm_tune_save(const char* path) {
    clear_error();
    if (!path || !*path) return fail(PERMX_EINVAL, "NULL or empty path");
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return fail(PERMX_EIO, "cannot open the tuning file for writing");
    bool ok = std::fprintf(f, "permx-tune 1\n") > 0;
    for (int field = 0; field < 3 && ok; ++field)
        for (int n = 1; n <= PERMX_MAX_N_MODP && ok; ++n) {
            const int t = tune_get(field, n);
            if (t > 0) ok = std::fprintf(f, "%d %d %d\n", field, n, t) > 0;
        }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(PERMX_EIO, "cannot write the tuning file");
    }
    return PERMX_OK;
}

int perm_tune_load(const char* path) {
    clear_error();
    if (!path || !*path) return fail(PERMX_EINVAL, "NULL or empty path");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(PERMX_EIO, "cannot open the tuning file");
    int table[3][PERMX_MAX_N_MODP + 1] = {};
    char line[256];
    int rc = PERMX_OK, lineno = 0;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        if (!std::strchr(line, '\n') && !std::feof(f)) {
            rc = fail(PERMX_EINVAL, "tuning file: line too long");
            break;
        }
        if (lineno == 1) {
            if (std::strcmp(line, "permx-tune 1\n") != 0 && std::strcmp(line, "permx-tune 1") != 0) {
                rc = fail(PERMX_EINVAL, "tuning file: missing 'permx-tune 1' header");
                break;
            }
            continue;
        }
        int field = -1, n = 0, ell = -1, used = 0;
        if (std::sscanf(line, "%d %d %d %n", &field, &n, &ell, &used) != 3 || line[used] != '\0' ||
            field < 0 || field > 2 || n < 1 || n > PERMX_MAX_N_MODP || ell < 1 ||
            ell > (field == PERMX_FIELD_MODP ? PERMX_MAX_ELL_MODP : PERMX_MAX_ELL_FP) || table[field][n]) {
            rc = fail(PERMX_EINVAL, "tuning file: bad or repeated entry on line " + std::to_string(lineno));
            break;
        }
        table[field][n] = ell;
    }
    if (rc == PERMX_OK && lineno == 0) rc = fail(PERMX_EINVAL, "tuning file: empty");
    if (rc == PERMX_OK && std::ferror(f)) rc = fail(PERMX_EIO, "cannot read the tuning file");
    std::fclose(f);
    if (rc) return rc;
    for (int field = 0; field < 3; ++field)
        for (int n = 1; n <= PERMX_MAX_N_MODP; ++n) tune_set(field, n, table[field][n]);
    return PERMX_OK;
}

int perm_autotune(int field, int32_t n, int64_t batch, int32_t reps, int32_t* best_ell) {
    clear_error();
    int rc = check_field(field);
    if (rc) return rc;
    const int maxn = field == PERMX_FIELD_MODP ? PERMX_MAX_N_MODP : PERMX_MAX_N_FP;
    if (n < 1 || n > maxn || batch < 1 || reps < 1 || !best_ell) return fail(PERMX_EINVAL, "bad arguments");
    const int bits = walk_bits(n, 1);
    const int saved = tune_get(field, n);
    tune_set(field, n, 0);
    const int ell0 = chunk_log2((Field)field, n, bits);
    const uint32_t prime = 2147483629u;
    const int entry_words = field == PERMX_FIELD_C128 ? 2 : 1;   // 8-byte words per entry (modp: 2 per word pair)
    const int64_t words = field == PERMX_FIELD_MODP ? ((int64_t)batch * n * n + 1) / 2
                                                    : (int64_t)batch * n * n * entry_words;
    std::vector<int32_t> nn(batch, n);
    std::vector<int64_t> off(batch);
    std::vector<uint32_t> pp(batch, prime);
    for (int64_t b = 0; b < batch; ++b) off[b] = b * (int64_t)n * n;
    cudaStream_t s;
    PERMX_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    void* A = nullptr;
    void* out = nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = ws_alloc(&A, 8 * (size_t)(words + 2), s);
    if (e == cudaSuccess) e = ws_alloc(&out, 16 * (size_t)batch, s);
    if (e == cudaSuccess) {
        tune_fill_kernel<<<256, 256, 0, s>>>(static_cast<unsigned long long*>(A), words, prime, field);
        e = cudaGetLastError();
    }
    float best_ms = 1e30f;
    int best = ell0;
    rc = e == cudaSuccess ? PERMX_OK : cuda_fail(e, "autotune set-up");
    for (int ell = std::max(1, ell0 - 3); rc == PERMX_OK && ell <= std::min(bits, ell0 + 3); ++ell) {
        tune_set(field, n, ell);
        Prepared X;
        rc = prepare_batch((Field)field, nn.data(), off.data(), pp.data(), batch, s, X);
        if (rc) break;
        rc = execute_batch(X, A, out, s);   // warm-up
        // each repetition timed on its own; the candidate's time is the fastest
        // one (interference from other work only ever adds time)
        float ms = 1e30f;
        for (int r = 0; rc == PERMX_OK && r < reps; ++r) {
            cudaEventRecord(e0, s);
            rc = execute_batch(X, A, out, s);
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            if (rc == PERMX_OK && e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
            float t = 0.f;
            if (rc == PERMX_OK) cudaEventElapsedTime(&t, e0, e1);
            if (rc == PERMX_OK && t < ms) ms = t;
        }
        release_batch(X, s);
        if (rc == PERMX_OK && ms < best_ms) {
            best_ms = ms;
            best = ell;
        }
    }
    ws_free(A, s);
    ws_free(out, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        tune_set(field, n, saved);
        return rc;
    }
    tune_set(field, n, best);
    *best_ell = best;
    return PERMX_OK;
}

}  // extern "C"
