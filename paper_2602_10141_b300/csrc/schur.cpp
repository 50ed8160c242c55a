// Exact perm(S_n) by F_p Ryser + CRT with checkpointed progress (paper §2.1
// method, §2.2 Gray-code blocks; long runs such as n = 43 take many slices).
//
// For every prime (the main primes, then one check prime) the residue matrix
// (g^{jk} mod p) is staged once; the Gray-index range [0, 2^n) is then walked
// in slices of whole chunks.  After every slice the running residue and the
// cursor are written to the checkpoint file (temp file + rename), so a killed
// process resumes at the last finished slice.
#include <cuda_runtime.h>

#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "field.h"
#include "schur.h"

namespace permx {

// ---------------------------------------------------------------------------
// single-matrix F_p range runner
// ---------------------------------------------------------------------------
int ModpRange::init(const uint32_t* A_dev, int n_, uint32_t p_, int nw_, cudaStream_t s_, uint64_t window) {
    n = n_;
    p = p_;
    s = s_;
    nw = nw_;
    bits = walk_bits(n, nw);
    ell = chunk_log2_modp(bits);
    if (window > 0) {
        int lw = 0;
        while (lw < 63 && (2ull << lw) <= window) ++lw;   // floor(log2(window))
        int cap = lw - 19;
        if (cap < 8) cap = 8;
        if (ell > cap) ell = cap;
    }
    ld = pad4(n);
    const size_t words = (size_t)(n + nw) * ld;
    PERMX_CUDA(ws_alloc(reinterpret_cast<void**>(&col), sizeof(uint32_t) * words + 256, s));
    acc = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(col) + ((sizeof(uint32_t) * words + 15) & ~size_t(15)));
    PERMX_CUDA(ws_alloc(reinterpret_cast<void**>(&params), 256, s));
    const uint32_t hp[2] = {p, inv_mod_2_32(p)};
    PERMX_CUDA(cudaMemcpyAsync(params, hp, sizeof hp, cudaMemcpyHostToDevice, s));
    PERMX_CUDA(stage_columns_u32(A_dev, n, ld, p, nw, col, s));
    return PERMX_OK;
}

int ModpRange::run(uint64_t k0, uint64_t k1, uint32_t* residue) {
    // residue = sum_{k0<=k<k1} (-1)^k prod_i r_i(S_k)  mod p, with r_i(S) = sum_{j in S} a_ij
    // (plus x_i in the Nijenhuis-Wilf form); no sign or factor of the formula applied
    *residue = 0;
    if (k0 >= k1) return PERMX_OK;
    PERMX_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s));
    ModpLaunch L;
    L.colT = col;
    L.p = params;
    L.pinv = params + 1;
    L.acc = acc;
    L.mat_stride = 0;
    const uint64_t Lc = 1ull << ell;
    L.item_begin = (k0 / Lc) & ~uint64_t(31);
    L.item_end = (k1 + Lc - 1) / Lc;
    L.k_lo = k0;
    L.k_hi = k1;
    L.ell = ell;
    L.log2_chunks = bits - ell;
    L.nw = nw;
    PERMX_CUDA(dispatch_modp(n, L, s));
    unsigned long long h = 0;
    PERMX_CUDA(cudaMemcpyAsync(&h, acc, sizeof h, cudaMemcpyDeviceToHost, s));
    PERMX_CUDA(cudaStreamSynchronize(s));
    const uint32_t rfix = pow_mod((uint32_t)((1ull << 32) % p), (uint64_t)(n - 1), p);
    *residue = (uint32_t)((h % p) * (uint64_t)rfix % p);
    return PERMX_OK;
}

void ModpRange::release() {
    if (col) ws_free(col, s);
    if (params) ws_free(params, s);
    col = nullptr;
    params = nullptr;
    acc = nullptr;
}

// ---------------------------------------------------------------------------
// checkpoint file
// ---------------------------------------------------------------------------
static uint64_t fnv1a(const std::string& s) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

static std::string ckpt_body(const SchurState& st) {
    std::string b = "permx-schur-ckpt 2\n";
    b += "n " + std::to_string(st.n) + "\n";
    b += "primes " + std::to_string(st.primes.size());
    for (uint32_t p : st.primes) b += " " + std::to_string(p);
    b += "\ndone " + std::to_string(st.done.size());
    for (uint32_t r : st.done) b += " " + std::to_string(r);
    b += "\ncursor " + std::to_string(st.cursor) + " " + std::to_string(st.partial) + "\n";
    return b;
}

int write_checkpoint(const std::string& path, const SchurState& st) {
    std::string body = ckpt_body(st);
    char tail[64];
    std::snprintf(tail, sizeof tail, "sum %016llx\n", (unsigned long long)fnv1a(body));
    body += tail;
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(PERMX_EIO, "cannot open checkpoint " + tmp + ": " + std::strerror(errno));
    // on disk before the rename makes it the checkpoint, so a crash leaves the
    // old file or the new one, never a truncated one
    bool ok = std::fwrite(body.data(), 1, body.size(), f) == body.size() && std::fflush(f) == 0 &&
              fsync(fileno(f)) == 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
        std::remove(tmp.c_str());
        return fail(PERMX_EIO, "cannot write checkpoint " + path);
    }
    return PERMX_OK;
}

// 1 = loaded, 0 = no file, <0 = error (corrupt or mismatched)
int read_checkpoint(const std::string& path, SchurState& st) {
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) {
        if (errno == ENOENT) return 0;
        return fail(PERMX_EIO, "cannot read checkpoint " + path + ": " + std::strerror(errno));
    }
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    const size_t pos = text.rfind("sum ");
    if (pos == std::string::npos) return fail(PERMX_EIO, "checkpoint " + path + " has no checksum");
    const std::string body = text.substr(0, pos);
    unsigned long long sum = 0;
    if (std::sscanf(text.c_str() + pos, "sum %llx", &sum) != 1 || sum != fnv1a(body))
        return fail(PERMX_EIO, "checkpoint " + path + " is corrupt (checksum mismatch)");
    SchurState r;
    const char* c = body.c_str();
    int used = 0, np = 0, nd = 0;
    if (std::sscanf(c, "permx-schur-ckpt 2\nn %d\nprimes %d%n", &r.n, &np, &used) != 2 || np < 1 ||
        np > PERMX_MAX_PRIMES + 1)
        return fail(PERMX_EIO, "checkpoint " + path + " has a bad header");
    c += used;
    for (int i = 0; i < np; ++i) {
        unsigned v;
        if (std::sscanf(c, " %u%n", &v, &used) != 1) return fail(PERMX_EIO, "checkpoint: bad prime list");
        r.primes.push_back(v);
        c += used;
    }
    if (std::sscanf(c, "\ndone %d%n", &nd, &used) != 1 || nd < 0 || nd > np)
        return fail(PERMX_EIO, "checkpoint: bad done list");
    c += used;
    for (int i = 0; i < nd; ++i) {
        unsigned v;
        if (std::sscanf(c, " %u%n", &v, &used) != 1) return fail(PERMX_EIO, "checkpoint: bad residue list");
        r.done.push_back(v);
        c += used;
    }
    unsigned long long cur = 0;
    unsigned part = 0;
    if (std::sscanf(c, "\ncursor %llu %u", &cur, &part) != 2) return fail(PERMX_EIO, "checkpoint: bad cursor");
    r.cursor = cur;
    r.partial = part;
    st = r;
    return 1;
}

// ---------------------------------------------------------------------------
// the run: primes, checkpointed slices, CRT
// ---------------------------------------------------------------------------
int schur_crt_run(int n, int nprimes, const char* ckpt_path, uint64_t slice_subsets, int64_t max_slices,
                  SchurResult& res) {
    if (n < 1 || n > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "n outside [1, 48]");
    if (nprimes < 0 || nprimes > PERMX_MAX_PRIMES - 1) return fail(PERMX_EINVAL, "nprimes outside [0, 63]");
    const int k = nprimes ? nprimes : schur_prime_count(n);
    std::vector<uint32_t> primes(k + 1);
    if (primes_1_mod_n(n, k + 1, 0, primes.data()) != k + 1) return fail(PERMX_EINVAL, "not enough primes");
    return schur_crt_run_primes(n, primes, ckpt_path, slice_subsets, max_slices, res);
}

int schur_crt_run_primes(int n, const std::vector<uint32_t>& primes, const char* ckpt_path, uint64_t slice_subsets,
                         int64_t max_slices, SchurResult& res) {
    if (n < 1 || n > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "n outside [1, 48]");
    if (primes.size() < 2 || primes.size() > (size_t)PERMX_MAX_PRIMES)
        return fail(PERMX_EINVAL, "need 2..64 primes (the last one checks)");
    for (size_t i = 0; i < primes.size(); ++i) {
        const uint32_t p = primes[i];
        if (p <= 2 || p >= (1u << 31) || !is_prime_u32(p) || p % (uint32_t)n != 1 % (uint32_t)n)
            return fail(PERMX_EINVAL, "prime " + std::to_string(p) + " is not an odd prime below 2^31 with p = 1 (mod n)");
        for (size_t j = 0; j < i; ++j)
            if (primes[j] == p) return fail(PERMX_EINVAL, "repeated prime " + std::to_string(p));
    }
    const int k = (int)primes.size() - 1;
    if (!modulus_suffices(n, primes.data(), k))
        return fail(PERMX_EINVAL, "product of " + std::to_string(k) + " primes does not exceed 2 n^(n/2)");

    SchurState st;
    st.n = n;
    st.primes = primes;
    const std::string path = ckpt_path ? ckpt_path : "";
    if (!path.empty()) {
        SchurState old;
        int rc = read_checkpoint(path, old);
        if (rc < 0) return rc;
        if (rc == 1) {
            if (old.n != n || old.primes != primes)
                return fail(PERMX_EINVAL, "checkpoint " + path + " belongs to a different run (n or primes differ)");
            st = old;
        }
    }

    // Nijenhuis-Wilf form: 2^(n-1) Gray indices per prime
    const uint64_t total = 1ull << walk_bits(n, 1);
    // a checkpoint whose checksum holds can still carry values no run writes:
    // reject them before any GPU work (a cursor at or past the end would never
    // advance, a residue at or above its prime would corrupt the CRT)
    for (size_t i = 0; i < st.done.size(); ++i)
        if (st.done[i] >= primes[i]) return fail(PERMX_EIO, "checkpoint " + path + ": residue not below its prime");
    if (st.done.size() < primes.size()) {
        if (st.cursor >= total) return fail(PERMX_EIO, "checkpoint " + path + ": cursor past the end of the walk");
        if (st.partial >= primes[st.done.size()])
            return fail(PERMX_EIO, "checkpoint " + path + ": partial sum not below its prime");
    } else if (st.cursor != 0 || st.partial != 0) {
        return fail(PERMX_EIO, "checkpoint " + path + ": finished run with a cursor");
    }
    const int ell = chunk_log2_modp(walk_bits(n, 1));
    uint64_t slice = slice_subsets ? slice_subsets : (n <= 38 ? total : (1ull << 37));
    const uint64_t Lc = 1ull << ell;
    slice = (slice + Lc - 1) / Lc * Lc;

    cudaStream_t s;
    PERMX_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    uint32_t* dA = nullptr;
    cudaError_t e = ws_alloc(reinterpret_cast<void**>(&dA), sizeof(uint32_t) * n * n, s);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return cuda_fail(e, "cudaMallocAsync");
    }
    std::vector<uint32_t> hA((size_t)n * n);
    int rc = PERMX_OK;
    int64_t slices = 0;
    while (st.done.size() < primes.size()) {
        const uint32_t p = primes[st.done.size()];
        uint32_t g = 0;
        if (primitive_root(p, n, &g) != 0) { rc = fail(PERMX_EINVAL, "no primitive root"); break; }
        schur_residues(n, p, g, hA.data());
        e = cudaMemcpyAsync(dA, hA.data(), sizeof(uint32_t) * n * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync"); break; }
        ModpRange R;
        rc = R.init(dA, n, p, 1, s, slice);
        while (rc == PERMX_OK && st.cursor < total) {
            if (max_slices > 0 && slices >= max_slices) { rc = PERMX_EAGAIN; break; }
            const uint64_t next = st.cursor + slice < total ? st.cursor + slice : total;
            uint32_t part = 0;
            rc = R.run(st.cursor, next, &part);
            if (rc) break;
            st.partial = (uint32_t)(((uint64_t)st.partial + part) % p);
            st.cursor = next;
            ++slices;
            if (st.cursor == total) {
                // perm = (-1)^(n-1) 2 sum
                const uint32_t v = (uint32_t)((uint64_t)st.partial * 2 % p);
                st.done.push_back((n & 1) ? v : (v ? p - v : 0));
                st.cursor = 0;
                st.partial = 0;
            }
            if (!path.empty()) {
                int wc = write_checkpoint(path, st);
                if (wc) { rc = wc; break; }
            }
            if (st.cursor == 0) break;   // this prime is finished
        }
        R.release();
        if (rc) break;
    }
    ws_free(dA, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc == PERMX_EAGAIN) return fail(PERMX_EAGAIN, "stopped after the requested number of slices");
    if (rc) return rc;

    Big mag;
    bool neg = false;
    crt_garner(st.done.data(), primes.data(), k, mag, neg);
    // the check prime
    const uint32_t pc = primes[k];
    uint32_t xm = mag.mod(pc);
    if (neg && xm) xm = pc - xm;
    res.primes = primes;
    res.residues = st.done;
    res.negative = neg;
    res.magnitude = mag;
    if (xm != st.done[k])
        return fail(PERMX_EIO, "CRT cross-check failed: the check prime's residue disagrees with the reconstruction");
    return PERMX_OK;
}

// One shard of a strong split of perm(S_n) over several GPUs: the
// Nijenhuis-Wilf walk of every prime is cut into `slices` equal Gray ranges;
// work item w = i * slices + j (prime i, range j) belongs to shard w mod
// nshards.  partial[i] = this shard's signed sum over its ranges of prime i
// mod p_i (0 if it has none), without the factor 2 (-1)^(n-1).
int schur_shard(int n, const std::vector<uint32_t>& primes, int slices, int shard, int nshards,
                std::vector<uint32_t>& partial) {
    if (n < 1 || n > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "n outside [1, 48]");
    if (primes.empty() || primes.size() > (size_t)PERMX_MAX_PRIMES) return fail(PERMX_EINVAL, "need 1..64 primes");
    if (slices < 1 || nshards < 1 || shard < 0 || shard >= nshards)
        return fail(PERMX_EINVAL, "need slices >= 1 and 0 <= shard < nshards");
    for (size_t i = 0; i < primes.size(); ++i) {
        const uint32_t p = primes[i];
        if (p <= 2 || p >= (1u << 31) || !is_prime_u32(p) || p % (uint32_t)n != 1 % (uint32_t)n)
            return fail(PERMX_EINVAL, "prime " + std::to_string(p) + " is not an odd prime below 2^31 with p = 1 (mod n)");
    }
    const uint64_t total = 1ull << walk_bits(n, 1);
    const uint64_t len = (total + (uint64_t)slices - 1) / (uint64_t)slices;
    partial.assign(primes.size(), 0);
    cudaStream_t s;
    PERMX_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    uint32_t* dA = nullptr;
    cudaError_t e = ws_alloc(reinterpret_cast<void**>(&dA), sizeof(uint32_t) * n * n, s);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return cuda_fail(e, "cudaMallocAsync");
    }
    std::vector<uint32_t> hA((size_t)n * n);
    int rc = PERMX_OK;
    for (size_t i = 0; i < primes.size() && rc == PERMX_OK; ++i) {
        std::vector<uint64_t> mine;
        for (int j = 0; j < slices; ++j)
            if (((uint64_t)i * (uint64_t)slices + (uint64_t)j) % (uint64_t)nshards == (uint64_t)shard) mine.push_back(j);
        if (mine.empty()) continue;
        const uint32_t p = primes[i];
        uint32_t g = 0;
        if (primitive_root(p, n, &g) != 0) { rc = fail(PERMX_EINVAL, "no primitive root"); break; }
        schur_residues(n, p, g, hA.data());
        e = cudaMemcpyAsync(dA, hA.data(), sizeof(uint32_t) * n * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync"); break; }
        ModpRange R;
        rc = R.init(dA, n, p, 1, s, len);
        for (size_t q = 0; q < mine.size() && rc == PERMX_OK; ++q) {
            const uint64_t k0 = mine[q] * len, k1 = k0 + len < total ? k0 + len : total;
            if (k0 >= k1) continue;
            uint32_t part = 0;
            rc = R.run(k0, k1, &part);
            if (rc == PERMX_OK) partial[i] = (uint32_t)(((uint64_t)partial[i] + part) % p);
        }
        R.release();
    }
    ws_free(dA, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return rc;
}

}  // namespace permx
