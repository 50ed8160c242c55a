// The C-ABI (include/permx.h): argument checks, error strings and the thin
// host wrappers around the batched, range and Schur drivers.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "field.h"
#include "schur.h"

namespace permx {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? PERMX_ENOMEM : PERMX_ECUDA;
}

static bool prime_ok(uint32_t p) { return p > 2 && p < (1u << 31) && is_prime_u32(p); }

static int check_primes(const uint32_t* p, int64_t batch) {
    if (!p) return fail(PERMX_EINVAL, "NULL prime array");
    uint32_t last = 0;
    for (int64_t b = 0; b < batch; ++b) {
        if (p[b] == last) continue;
        if (!prime_ok(p[b]))
            return fail(PERMX_EINVAL, "p[" + std::to_string(b) + "] = " + std::to_string(p[b]) +
                                          " is not an odd prime below 2^31");
        last = p[b];
    }
    return PERMX_OK;
}

static void write_i128(const Big& mag, bool neg, int64_t out[2], bool& fits) {
    // two's complement of +-mag in 128 bits
    unsigned __int128 m = 0;
    fits = mag.w.size() <= 4;
    for (size_t i = 0; i < mag.w.size() && i < 4; ++i) m |= (unsigned __int128)mag.w[i] << (32 * i);
    if (fits) fits = neg ? m <= ((unsigned __int128)1 << 127) : m < ((unsigned __int128)1 << 127);
    unsigned __int128 v = neg ? (unsigned __int128)0 - m : m;
    out[0] = (int64_t)(uint64_t)v;
    out[1] = (int64_t)(uint64_t)(v >> 64);
}

// host-buffer variants: copy in, run, copy out, synchronise
template <typename T, typename F>
static int host_call(const T* A, const int32_t* n, const int64_t* offset, int64_t batch, T* out, void* stream,
                     int max_n, F&& run) {
    clear_error();
    int rc = validate_batch(A, n, offset, batch, out, max_n);
    if (rc || batch == 0) return rc;
    int64_t elems = 0;
    for (int64_t b = 0; b < batch; ++b) {
        const int64_t end = offset[b] + (int64_t)n[b] * n[b];
        if (end > elems) elems = end;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    T* dA = nullptr;
    T* dO = nullptr;
    PERMX_CUDA(ws_alloc(reinterpret_cast<void**>(&dA), sizeof(T) * (size_t)elems, s));
    cudaError_t e = ws_alloc(reinterpret_cast<void**>(&dO), sizeof(T) * (size_t)batch, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dA, A, sizeof(T) * (size_t)elems, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        ws_free(dA, s);
        if (dO) ws_free(dO, s);
        return cuda_fail(e, "host copy-in");
    }
    rc = run(dA, dO, s);
    if (rc == PERMX_OK) {
        e = cudaMemcpyAsync(out, dO, sizeof(T) * (size_t)batch, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "host copy-out");
    }
    ws_free(dA, s);
    ws_free(dO, s);
    e = cudaStreamSynchronize(s);
    if (rc == PERMX_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

}  // namespace permx

using namespace permx;

extern "C" {

const char* perm_last_error(void) { return g_last_error.c_str(); }
const char* permx_version(void) { return "permx 0.1 (sm_103a)"; }

int perm_c128(const perm_c128_t* A, const int32_t* n, const int64_t* offset, int64_t batch, perm_c128_t* out,
              void* stream) {
    clear_error();
    int rc = validate_batch(A, n, offset, batch, out, PERMX_MAX_N_FP);
    if (rc || batch == 0) return rc;
    if (reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(out) % 16)
        return fail(PERMX_EINVAL, "complex128 arrays must be 16-byte aligned");
    return run_fp_batch(reinterpret_cast<const double*>(A), n, offset, batch, out, true,
                        static_cast<cudaStream_t>(stream));
}

int perm_f64(const double* A, const int32_t* n, const int64_t* offset, int64_t batch, double* out, void* stream) {
    clear_error();
    int rc = validate_batch(A, n, offset, batch, out, PERMX_MAX_N_FP);
    if (rc || batch == 0) return rc;
    return run_fp_batch(A, n, offset, batch, out, false, static_cast<cudaStream_t>(stream));
}

int perm_modp(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
              uint32_t* out, void* stream) {
    clear_error();
    int rc = validate_batch(A, n, offset, batch, out, PERMX_MAX_N_MODP);
    if (rc || batch == 0) return rc;
    rc = check_primes(p, batch);
    if (rc) return rc;
    return run_modp_batch(A, n, offset, p, batch, out, static_cast<cudaStream_t>(stream));
}

int perm_c128_host(const perm_c128_t* A, const int32_t* n, const int64_t* offset, int64_t batch, perm_c128_t* out,
                   void* stream) {
    return host_call(A, n, offset, batch, out, stream, PERMX_MAX_N_FP,
                     [&](const perm_c128_t* dA, perm_c128_t* dO, cudaStream_t s) {
                         return run_fp_batch(reinterpret_cast<const double*>(dA), n, offset, batch, dO, true, s);
                     });
}

int perm_f64_host(const double* A, const int32_t* n, const int64_t* offset, int64_t batch, double* out,
                  void* stream) {
    return host_call(A, n, offset, batch, out, stream, PERMX_MAX_N_FP,
                     [&](const double* dA, double* dO, cudaStream_t s) {
                         return run_fp_batch(dA, n, offset, batch, dO, false, s);
                     });
}

int perm_modp_host(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                   uint32_t* out, void* stream) {
    clear_error();
    int rc = validate_batch(A, n, offset, batch, out, PERMX_MAX_N_MODP);
    if (rc || batch == 0) return rc;
    rc = check_primes(p, batch);
    if (rc) return rc;
    for (int64_t b = 0; b < batch; ++b)
        for (int64_t e = 0; e < (int64_t)n[b] * n[b]; ++e)
            if (A[offset[b] + e] >= p[b])
                return fail(PERMX_EINVAL, "matrix " + std::to_string(b) + " has an entry >= p");
    return host_call(A, n, offset, batch, out, stream, PERMX_MAX_N_MODP,
                     [&](const uint32_t* dA, uint32_t* dO, cudaStream_t s) {
                         return run_modp_batch(dA, n, offset, p, batch, dO, s);
                     });
}

int perm_modp_gray_range(const uint32_t* A, int32_t n, uint32_t p, uint64_t k0, uint64_t k1, uint32_t* out,
                         void* stream) {
    clear_error();
    if (!A || !out) return fail(PERMX_EINVAL, "NULL pointer argument");
    if (n < 1 || n > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "n outside [1, 48]");
    if (!prime_ok(p)) return fail(PERMX_EINVAL, "p is not an odd prime below 2^31");
    if (k0 > k1 || k1 > (1ull << n)) return fail(PERMX_EINVAL, "need k0 <= k1 <= 2^n");
    ModpRange R;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = R.init(A, n, p, 0, s, k1 - k0);   // plain Ryser: the range is over subsets of all n columns
    if (rc == PERMX_OK) rc = R.run(k0, k1, out);
    R.release();
    cudaError_t e = cudaStreamSynchronize(s);
    if (rc == PERMX_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

}  // extern "C"

namespace permx {
static int schur_outputs(int rc, const SchurResult& res, int64_t out_i128[2], char* out_dec, size_t out_dec_len,
                         uint32_t* residues_out, uint32_t* primes_out);
}  // namespace permx

extern "C" {

int perm_schur_crt_primes(int32_t n, const uint32_t* primes, int32_t count, const char* ckpt_path,
                          uint64_t slice_subsets, int64_t max_slices, int64_t out_i128[2], char* out_dec,
                          size_t out_dec_len, uint32_t* residues_out) {
    clear_error();
    if (!out_i128 && !out_dec) return fail(PERMX_EINVAL, "no output buffer");
    if (!primes || count < 2 || count > PERMX_MAX_PRIMES) return fail(PERMX_EINVAL, "need 2..64 primes");
    SchurResult res;
    const std::vector<uint32_t> pv(primes, primes + count);
    const int rc = schur_crt_run_primes(n, pv, ckpt_path, slice_subsets, max_slices, res);
    return schur_outputs(rc, res, out_i128, out_dec, out_dec_len, residues_out, nullptr);
}

int perm_schur_shard(int32_t n, const uint32_t* primes, int32_t count, int32_t slices, int32_t shard, int32_t nshards,
                     uint32_t* partial_out) {
    clear_error();
    if (!primes || !partial_out || count < 1 || count > PERMX_MAX_PRIMES) return fail(PERMX_EINVAL, "bad arguments");
    std::vector<uint32_t> part;
    const int rc = schur_shard(n, std::vector<uint32_t>(primes, primes + count), slices, shard, nshards, part);
    if (rc) return rc;
    for (int32_t i = 0; i < count; ++i) partial_out[i] = part[(size_t)i];
    return PERMX_OK;
}

int perm_schur_crt_ex(int32_t n, int32_t nprimes, const char* ckpt_path, uint64_t slice_subsets, int64_t max_slices,
                      int64_t out_i128[2], char* out_dec, size_t out_dec_len, uint32_t* residues_out,
                      uint32_t* primes_out) {
    clear_error();
    if (!out_i128 && !out_dec) return fail(PERMX_EINVAL, "no output buffer");
    SchurResult res;
    const int rc = schur_crt_run(n, nprimes, ckpt_path, slice_subsets, max_slices, res);
    return schur_outputs(rc, res, out_i128, out_dec, out_dec_len, residues_out, primes_out);
}

}  // extern "C"

namespace permx {
static int schur_outputs(int rc, const SchurResult& res, int64_t out_i128[2], char* out_dec, size_t out_dec_len,
                         uint32_t* residues_out, uint32_t* primes_out) {
    if (residues_out)
        for (size_t i = 0; i < res.residues.size(); ++i) residues_out[i] = res.residues[i];
    if (primes_out)
        for (size_t i = 0; i < res.primes.size(); ++i) primes_out[i] = res.primes[i];
    if (rc) return rc;
    const std::string dec = (res.negative ? "-" : "") + res.magnitude.decimal();
    bool fits = false;
    int64_t tmp[2];
    write_i128(res.magnitude, res.negative, tmp, fits);
    if (out_i128) {
        if (!fits) return fail(PERMX_EINVAL, "perm(S_n) = " + dec + " does not fit in 128 bits; use out_dec");
        out_i128[0] = tmp[0];
        out_i128[1] = tmp[1];
    }
    if (out_dec) {
        if (out_dec_len < dec.size() + 1) return fail(PERMX_EINVAL, "out_dec too small");
        std::memcpy(out_dec, dec.c_str(), dec.size() + 1);
    }
    return PERMX_OK;
}
}  // namespace permx

extern "C" {

int perm_schur_crt(int32_t n, int32_t nprimes, const char* ckpt_path, int64_t out_i128[2], char* out_dec,
                   size_t out_dec_len) {
    return perm_schur_crt_ex(n, nprimes, ckpt_path, 0, 0, out_i128, out_dec, out_dec_len, nullptr, nullptr);
}

int perm_primes_1_mod_n(int32_t n, int32_t count, int32_t skip, uint32_t* primes_out) {
    clear_error();
    if (n < 1 || count < 0 || skip < 0 || (!primes_out && count > 0)) return fail(PERMX_EINVAL, "bad arguments");
    const int got = primes_1_mod_n(n, count, skip, primes_out);
    if (got != count) return fail(PERMX_EINVAL, "not enough primes below 2^31");
    return got;
}

int perm_primitive_root(uint32_t p, int32_t n, uint32_t* g_out) {
    clear_error();
    if (!g_out || !prime_ok(p) || n < 1 || (p - 1) % (uint32_t)n) return fail(PERMX_EINVAL, "need prime p = 1 mod n");
    if (primitive_root(p, n, g_out) != 0) return fail(PERMX_EINVAL, "no primitive root");
    return PERMX_OK;
}

int perm_schur_residues(int32_t n, uint32_t p, uint32_t g, uint32_t* out) {
    clear_error();
    if (!out || n < 1 || n > PERMX_MAX_N_MODP || !prime_ok(p) || g == 0 || g >= p)
        return fail(PERMX_EINVAL, "bad arguments");
    schur_residues(n, p, g, out);
    return PERMX_OK;
}

int perm_crt(const uint32_t* residues, const uint32_t* primes, int32_t k, int64_t out_i128[2]) {
    clear_error();
    if (!residues || !primes || !out_i128 || k < 1 || k > PERMX_MAX_PRIMES) return fail(PERMX_EINVAL, "bad arguments");
    for (int i = 0; i < k; ++i) {
        if (!prime_ok(primes[i]) || residues[i] >= primes[i]) return fail(PERMX_EINVAL, "bad prime or residue");
        for (int j = 0; j < i; ++j)
            if (primes[j] == primes[i]) return fail(PERMX_EINVAL, "primes must be distinct");
    }
    Big mag;
    bool neg = false;
    crt_garner(residues, primes, k, mag, neg);
    bool fits = false;
    write_i128(mag, neg, out_i128, fits);
    if (!fits) return fail(PERMX_EINVAL, "value does not fit in 128 bits");
    return PERMX_OK;
}

int permx_set_fp_arith(int mode) {
    clear_error();
    if (mode != PERMX_FP_ARITH_FP64 && mode != PERMX_FP_ARITH_INT)
        return fail(PERMX_EINVAL, "unknown float arithmetic mode");
    return set_fp_arith(mode);
}

int permx_get_fp_arith(void) { return fp_arith(); }

int perm_schur_prime_count(int32_t n) {
    clear_error();
    if (n < 1 || n > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "n outside [1, 48]");
    return schur_prime_count(n);
}

}  // extern "C"
