// Batched (ragged) permanents: planning, column-major staging, launches and
// fixed-order finalisation.  Entry points perm_modp / perm_f64 / perm_c128.
//
// A call groups the matrices by n (one compile-time kernel per n), stages each
// matrix column-major into a stream-ordered workspace (column j contiguous,
// padded to 16 bytes), launches one Ryser kernel per group and finishes with
// one finalize kernel for the whole batch.  Per-matrix results do not depend on
// the batch: the chunking is a function of (n, field) only and chunk partials
// are combined in a fixed order.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "finalize.cuh"
#include "pdl.cuh"
#include "x64_arith.cuh"

namespace permx {

int chunk_log2_modp(int bits) {
    // Enough chunks to fill the GPU for one large matrix (about 2^22 chunks),
    // at least 2^8 subsets per chunk so the O(n^2) chunk start stays < 1%.
    int ell = bits - 22;
    int lo = bits < 8 ? bits : 8;
    return ell < lo ? lo : ell;
}

// Tuning table: chunk length (log2) per (field, n) set by perm_tune_set /
// perm_autotune; 0 means the formula.  Float results depend on the chunking,
// so a given table always gives the same bits.
static std::atomic<int> g_tune[3][PERMX_MAX_N_MODP + 1];

int tune_get(int field, int n) {
    if (field < 0 || field > 2 || n < 1 || n > PERMX_MAX_N_MODP) return 0;
    return g_tune[field][n].load();
}
void tune_set(int field, int n, int ell) {
    if (field >= 0 && field <= 2 && n >= 1 && n <= PERMX_MAX_N_MODP) g_tune[field][n].store(ell);
}

int chunk_log2(Field field, int n, int bits) {
    const int t = tune_get((int)field, n);
    int ell = t > 0 ? (t < bits ? t : bits) : (field == Field::MODP ? chunk_log2_modp(bits) : chunk_log2_fp(bits));
    if (field == Field::MODP && ell > kModpMaxEll) ell = kModpMaxEll;   // the walk counts steps in 32 bits
    return ell;
}

int chunk_log2_fp(int bits) {
    // About 2^14 chunks per matrix (2^(bits-3) for small walks) so that even
    // one matrix spreads over many threads (a chunk's steps run serially, so
    // its length sets the latency of a lone matrix); at most 2^8 steps per
    // chunk (a chunk is the unit of work a serving step cannot split: 2^8
    // steps of a complex n = 26 walk take about 2 ms on one thread, and the
    // float64 walk's row-sum drift grows like sqrt(L) ulps), which costs
    // n^2 / (2^8 n) < 13 % extra row-sum work at n = 32; at least 2^3 steps
    // (or the whole walk), where the O(n^2) chunk start is still small next to
    // the n products per step.
    int ell = bits - 14;
    int lo = bits < 3 ? bits : 3;
    if (ell < lo) ell = lo;
    if (ell > 8) ell = 8;
    return ell;
}

// Stream-ordered workspace from a pool owned by the library (one per device),
// which keeps freed memory for reuse instead of returning it at every
// synchronisation; a batched call then costs no allocator round trip.
cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t ws_free(void* p, cudaStream_t s) { return p ? cudaFreeAsync(p, s) : cudaSuccess; }

static std::atomic<int> g_fp_arith{1};
int fp_arith() { return g_fp_arith.load(); }
int set_fp_arith(int mode) { return g_fp_arith.exchange(mode); }

int sm_count() {
    static std::atomic<int> cached[64];   // zero-initialised (static storage)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// ---------------------------------------------------------------------------
// device kernels: staging and finalisation
// ---------------------------------------------------------------------------

// Integer-mantissa staging of one matrix by one block: row i gets the scale
// sigma_i = 62 - floor(log2(sum_j |a_ij|)) (complex: |re| + |im|), entries
// A_ij = 2 round(a_ij 2^(sigma_i - 1)) (even, so halves are exact), the
// Nijenhuis-Wilf column X_i = A_{i,n-1}/2 - sum_{j<n-1} A_ij/2, zero padding,
// and one trailing word with -sum_i sigma_i.  W = int64 words per entry.  The
// matrix is read once into shared memory; the row scales take one thread per
// row (the float sum as four interleaved partial sums), the conversions one
// thread per entry, in integer operations.
constexpr int kStageX64Threads = 128;
struct NoWork {
    __device__ void operator()() const {}
};
// mid() runs while the matrix loads are in flight (the set-up kernel's
// metadata copy), before the first barrier.
template <int W, typename Mid = NoWork>
__device__ __forceinline__ void stage_x64_block(const double* __restrict__ A, const StageDesc s,
                                                int64_t* __restrict__ colT, Mid mid = Mid()) {
    // the matrix, row-major: the float entries, each replaced in place by its
    // integer A_ij once the row scales are known
    __shared__ long long buf[PERMX_MAX_N_FP * PERMX_MAX_N_FP * W];
    __shared__ int sig_row[PERMX_MAX_N_FP];   // sigma_i, or kNonFinite
    __shared__ int sig_sum, bad;
    constexpr int kNonFinite = -1 << 30;
    const int n = s.n, ld = s.ld, nw = n * W, tot = n * nw;
    int64_t* base = colT + s.dst * W;   // dst counts entries of W words
    const long long* src = reinterpret_cast<const long long*>(A + s.src * W);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) buf[e] = src[e];   // one coalesced pass
    if (threadIdx.x == 0) {
        sig_sum = 0;
        bad = 0;
    }
    mid();
    __syncthreads();
    // the row scale from sum_j |a_ij|, one thread per row: four interleaved
    // partial sums over the row's words (words 0, 4, 8, ... in s0), then
    // (s0 + s1) + (s2 + s3); FP64 latency on B300 is ~64 cycles per dependent
    // add, so a single running sum would dominate the staging
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const long long* row = buf + i * nw;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = 0;
        for (; j + 4 <= nw; j += 4) {
            s0 += fabs(__longlong_as_double(row[j]));
            s1 += fabs(__longlong_as_double(row[j + 1]));
            s2 += fabs(__longlong_as_double(row[j + 2]));
            s3 += fabs(__longlong_as_double(row[j + 3]));
        }
        if (j < nw) s0 += fabs(__longlong_as_double(row[j]));
        if (j + 1 < nw) s1 += fabs(__longlong_as_double(row[j + 1]));
        if (j + 2 < nw) s2 += fabs(__longlong_as_double(row[j + 2]));
        const double S = (s0 + s1) + (s2 + s3);
        // a NaN or infinite entry makes S non-finite: the matrix is flagged (its
        // permanent is reported as NaN) and the row staged as zeros
        const bool finite = isfinite(S);
        if (!finite) atomicOr(&bad, 1);
        const int sig = finite && S > 0.0 ? 62 - ilogb(S) : 0;
        sig_row[i] = finite ? sig : kNonFinite;
        atomicAdd(&sig_sum, sig);
    }
    __syncthreads();
    // entries, one thread each: A_ij = 2 round(a_ij 2^(sigma_i - 1))
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int i = e / nw, jw = e - i * nw, j = jw / W, w = jw - j * W;
        const int sig = sig_row[i];
        const int64_t a = sig != kNonFinite ? 2 * x64_scaled_round(__longlong_as_double(buf[e]), sig - 1) : 0;
        buf[e] = a;
        base[((int64_t)j * ld + i) * W + w] = a;
    }
    // padding rows n..ld-1 of every column, the x column included
    for (int e = threadIdx.x; e < (ld - n) * (n + 1) * W; e += blockDim.x) {
        const int q = e / W, w = e - q * W, j = q / (ld - n), i = n + (q - j * (ld - n));
        base[((int64_t)j * ld + i) * W + w] = 0;
    }
    __syncthreads();
    // the Nijenhuis-Wilf column X_i = A_{i,n-1} - (sum_j A_ij) / 2 = A_{i,n-1}/2 - sum_{j<n-1} A_ij/2,
    // exact (entries are even), summed in halves so no partial sum leaves int64
    for (int e = threadIdx.x; e < n * W; e += blockDim.x) {
        const int i = e / W, w = e - i * W;
        const long long* col0 = buf + i * nw + w;
        int64_t h0 = 0, h1 = 0, h2 = 0, h3 = 0;   // exact integer sums: the split changes no bit
        int j = 0;
        for (; j + 4 <= n - 1; j += 4) {
            h0 += col0[j * W] / 2;
            h1 += col0[(j + 1) * W] / 2;
            h2 += col0[(j + 2) * W] / 2;
            h3 += col0[(j + 3) * W] / 2;
        }
        if (j < n - 1) h0 += col0[j * W] / 2;
        if (j + 1 < n - 1) h1 += col0[(j + 1) * W] / 2;
        if (j + 2 < n - 1) h2 += col0[(j + 2) * W] / 2;
        const int64_t half = (h0 + h1) + (h2 + h3);
        base[((int64_t)n * ld + i) * W + w] = buf[i * nw + (n - 1) * W + w] / 2 - half;
    }
    if (threadIdx.x == 0) {
        base[(int64_t)(n + 1) * ld * W] = -(int64_t)sig_sum;
        base[(int64_t)(n + 1) * ld * W + 1] = bad;   // 1: non-finite entry, result NaN
    }
}

template <int W>
__global__ void __launch_bounds__(kStageX64Threads) stage_x64_kernel(const double* __restrict__ A,
                                                                   const StageDesc* __restrict__ d,
                                                                   int64_t* __restrict__ colT) {
    grid_dep_allow();
    stage_x64_block<W>(A, d[blockIdx.x], colT);
}

// x_i = a_{i,n-1} - (1/2) sum_j a_ij for the Nijenhuis-Wilf form.
// F_p: 1/2 = (p+1)/2 mod p.  Floating point: the row sum is compensated
// (Neumaier), the halving is exact.
__device__ __forceinline__ uint32_t x_entry(const uint32_t* __restrict__ row, int n, uint32_t p) {
    uint64_t s = 0;
    for (int j = 0; j < n; ++j) s += row[j];
    const uint64_t hs = (s % p) * (uint64_t)((p + 1) / 2) % p;
    return (uint32_t)(((uint64_t)row[n - 1] + p - hs) % p);
}
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}
__device__ __forceinline__ double x_entry(const double* __restrict__ row, int n, uint32_t) {
    double s = 0.0, c = 0.0;
    for (int j = 0; j < n; ++j) neumaier(s, c, row[j]);
    return row[n - 1] - 0.5 * (s + c);
}
__device__ __forceinline__ double2 x_entry(const double2* __restrict__ row, int n, uint32_t) {
    double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
    for (int j = 0; j < n; ++j) {
        neumaier(sr, cr, row[j].x);
        neumaier(si, ci, row[j].y);
    }
    return make_double2(row[n - 1].x - 0.5 * (sr + cr), row[n - 1].y - 0.5 * (si + ci));
}

// One block per matrix: colT[dst + j*ld + i] = A[src + i*n + j], padding
// zeroed, and in the Nijenhuis-Wilf form the x column at colT[dst + n*ld + i].
// A residue at or above p is taken mod p (the walk's modular adds assume
// [0, p)); float entries pass unchanged.
__device__ __forceinline__ uint32_t staged_entry(uint32_t v, uint32_t p) { return v < p ? v : v % p; }
__device__ __forceinline__ double staged_entry(double v, uint32_t) { return v; }
__device__ __forceinline__ double2 staged_entry(double2 v, uint32_t) { return v; }

template <typename T>
__device__ __forceinline__ void stage_columns_block(const T* __restrict__ A, const StageDesc s, T* __restrict__ colT) {
    const int n = s.n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        colT[s.dst + (int64_t)j * s.ld + i] = staged_entry(A[s.src + e], s.p);
    }
    for (int e = threadIdx.x; e < n * (s.ld - n); e += blockDim.x) {   // zero the padding
        const int j = e / (s.ld - n), i = n + e % (s.ld - n);
        colT[s.dst + (int64_t)j * s.ld + i] = T{};
    }
    if (s.nw)
        for (int i = threadIdx.x; i < s.ld; i += blockDim.x)
            colT[s.dst + (int64_t)n * s.ld + i] = i < n ? x_entry(A + s.src + (int64_t)i * n, n, s.p) : T{};
}

template <typename T>
__global__ void stage_columns_kernel(const T* __restrict__ A, const StageDesc* __restrict__ d, T* __restrict__ colT) {
    grid_dep_allow();
    stage_columns_block<T>(A, d[blockIdx.x], colT);
}

// Set-up of a call whose metadata is small enough to travel as a kernel
// parameter: block 0 writes the metadata into the workspace and clears the
// words that must start at zero (F_p accumulators, the groups' finalisation
// tickets); block b stages matrix b from its descriptor in the parameter.
// One launch where an upload and a staging launch would otherwise run.
template <int SZ>
struct alignas(16) MetaBytes {
    uint32_t words, pad_[3];
    uint32_t w[SZ / 4];        // 16-byte aligned: the descriptors read from it hold 8-byte fields
};
static_assert(offsetof(MetaBytes<1024>, w) % 16 == 0, "metadata words must be 16-byte aligned");
template <int SZ>
__device__ __forceinline__ void setup_meta(const MetaBytes<SZ>& m, uint32_t* __restrict__ dst, uint32_t zero_from,
                                           uint32_t zero_words) {
    if (blockIdx.x != 0) return;
    for (uint32_t i = threadIdx.x; i < m.words; i += blockDim.x) dst[i] = m.w[i];
    for (uint32_t i = threadIdx.x; i < zero_words; i += blockDim.x) dst[zero_from + i] = 0;
}
template <int SZ, typename T>
__global__ void setup_columns_kernel(const T* __restrict__ A, const __grid_constant__ MetaBytes<SZ> m,
                                     uint32_t* __restrict__ ws, uint32_t zero_from, uint32_t zero_words,
                                     T* __restrict__ colT) {
    grid_dep_allow();   // the walk may be scheduled now; it waits for this kernel (pdl.cuh)
    setup_meta(m, ws, zero_from, zero_words);
    stage_columns_block<T>(A, reinterpret_cast<const StageDesc*>(m.w)[blockIdx.x], colT);
}
template <int SZ, int W>
__global__ void __launch_bounds__(kStageX64Threads) setup_x64_kernel(const double* __restrict__ A,
                                                                   const __grid_constant__ MetaBytes<SZ> m,
                                                                   uint32_t* __restrict__ ws, uint32_t zero_from,
                                                                   uint32_t zero_words, int64_t* __restrict__ colT) {
    grid_dep_allow();   // the walk may be scheduled now; it waits for this kernel (pdl.cuh)
    stage_x64_block<W>(A, reinterpret_cast<const StageDesc*>(m.w)[blockIdx.x], colT,
                       [&] { setup_meta(m, ws, zero_from, zero_words); });
}

__global__ void finalize_modp_kernel(const unsigned long long* __restrict__ acc, const ModpFinal* __restrict__ f,
                                     int64_t count, uint32_t* __restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const ModpFinal x = f[b];
    out[x.out_index] = finalize_modp_value(acc[b], x);
}

// One block (kFinalThreads threads) per matrix: the fixed-order double-double
// sum of its partial slots (finalize_fp_block).
__global__ void __launch_bounds__(kFinalThreads) finalize_fp_kernel(const double* __restrict__ partial,
                                                                    const FpFinal* __restrict__ f,
                                                                    int cplx, void* __restrict__ out) {
    __shared__ double sh[4][kFinalThreads];
    finalize_fp_block(partial, f[blockIdx.x], cplx, out, sh);
}
// Integer mode: the XPart slots merged in integers, rounded once (finalize_x64_block).
__global__ void __launch_bounds__(kFinalThreads) finalize_x64_kernel(const XPart* __restrict__ partial,
                                                                     const FpFinal* __restrict__ f,
                                                                     int cplx, void* __restrict__ out) {
    __shared__ XFinSh sh;
    finalize_x64_block(partial, f[blockIdx.x], cplx, out, sh);
}

// Server variant: accumulators and outputs at arbitrary indices.
__global__ void finalize_modp_at_kernel(const unsigned long long* __restrict__ acc, const ModpFinalAt* __restrict__ f,
                                        int64_t count, uint32_t* __restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const ModpFinalAt x = f[b];
    const ModpFinal y{x.p, x.rfix, x.negate, 0, x.out_index};
    out[x.out_index] = finalize_modp_value(acc[x.acc_index], y);
}

cudaError_t launch_stage(int field, const void* A, const StageDesc* d, int64_t count, void* colT, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (field == (int)Field::MODP)
        stage_columns_kernel<uint32_t><<<(unsigned)count, 256, 0, s>>>(static_cast<const uint32_t*>(A), d,
                                                                         static_cast<uint32_t*>(colT));
    else if (field == (int)Field::F64)
        stage_columns_kernel<double><<<(unsigned)count, 256, 0, s>>>(static_cast<const double*>(A), d,
                                                                       static_cast<double*>(colT));
    else
        stage_columns_kernel<double2><<<(unsigned)count, 256, 0, s>>>(static_cast<const double2*>(A), d,
                                                                        static_cast<double2*>(colT));
    return cudaGetLastError();
}

cudaError_t launch_stage_x64(bool cplx, const void* A, const StageDesc* d, int64_t count, void* colT,
                             cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (cplx)
        stage_x64_kernel<2><<<(unsigned)count, kStageX64Threads, 0, s>>>(static_cast<const double*>(A), d,
                                                            static_cast<int64_t*>(colT));
    else
        stage_x64_kernel<1><<<(unsigned)count, kStageX64Threads, 0, s>>>(static_cast<const double*>(A), d,
                                                            static_cast<int64_t*>(colT));
    return cudaGetLastError();
}

cudaError_t launch_finalize_fp(const double* partial, const FpFinal* f, int64_t count, bool cplx, bool x64,
                               void* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (x64)
        finalize_x64_kernel<<<(unsigned)count, kFinalThreads, 0, s>>>(reinterpret_cast<const XPart*>(partial), f,
                                                                      cplx ? 1 : 0, out);
    else
        finalize_fp_kernel<<<(unsigned)count, kFinalThreads, 0, s>>>(partial, f, cplx ? 1 : 0, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize_modp_at(const unsigned long long* acc, const ModpFinalAt* f, int64_t count, uint32_t* out,
                                    cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    finalize_modp_at_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(acc, f, count, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// primes seen before (checked once per process)
std::mutex g_prime_mu;
std::vector<uint32_t> g_prime_ok;

bool checked_prime(uint32_t p) {
    {
        std::lock_guard<std::mutex> lk(g_prime_mu);
        if (std::find(g_prime_ok.begin(), g_prime_ok.end(), p) != g_prime_ok.end()) return true;
    }
    if (p <= 2 || p >= (1u << 31) || !is_prime_u32(p)) return false;
    std::lock_guard<std::mutex> lk(g_prime_mu);
    if (g_prime_ok.size() > 4096) g_prime_ok.clear();
    g_prime_ok.push_back(p);
    return true;
}

}  // namespace

int validate_batch(const void* A, const int32_t* n, const int64_t* offset, int64_t batch, const void* out,
                   int max_n) {
    if (batch < 0) return fail(PERMX_EINVAL, "batch < 0");
    if (batch == 0) return PERMX_OK;
    if (!A || !n || !offset || !out) return fail(PERMX_EINVAL, "NULL pointer argument");
    for (int64_t b = 0; b < batch; ++b) {
        if (n[b] < 1 || n[b] > max_n)
            return fail(PERMX_EINVAL, "n[" + std::to_string(b) + "] = " + std::to_string(n[b]) + " outside [1, " +
                                          std::to_string(max_n) + "]");
        if (offset[b] < 0) return fail(PERMX_EINVAL, "offset[" + std::to_string(b) + "] < 0");
    }
    return PERMX_OK;
}

BatchPlan plan_batch(const int32_t* n, int64_t batch, Field field) {
    BatchPlan P;
    P.field = field;
    std::map<int, std::vector<int64_t>> by_n;
    for (int64_t b = 0; b < batch; ++b) by_n[n[b]].push_back(b);
    int64_t col_off = 0, mat_index = 0, part_off = 0;
    for (auto& kv : by_n) {
        GroupPlan g;
        g.n = kv.first;
        g.mats = std::move(kv.second);
        g.nw = 1;
        const int bits = walk_bits(g.n, g.nw);
        g.ell = chunk_log2(field, g.n, bits);
        g.log2_chunks = bits - g.ell;
        if (field == Field::MODP) g.ld = pad4(g.n);
        else if (field == Field::F64) g.ld = pad2(g.n);
        else g.ld = g.n;                          // complex entries are 16 bytes already
        const int words = field == Field::C128 ? 2 : 1;   // doubles (fp) or uint32 (modp) per entry
        g.mat_stride = (int64_t)(g.n + g.nw) * g.ld * words;
        g.x64 = field != Field::MODP && fp_arith() == 1;
        if (g.x64) g.mat_stride += 2;             // the -sum(sigma) word (and padding)
        g.col_off = col_off;
        g.first_mat = mat_index;
        g.items = (int64_t)g.mats.size() << g.log2_chunks;
        const int lg = group_log2(g.log2_chunks, chunks_per_warp(g.x64, field == Field::C128, g.n));
        g.partials_per_mat = (int64_t)1 << (g.log2_chunks - lg);
        g.part_off = part_off;
        col_off += g.mat_stride * (int64_t)g.mats.size();
        mat_index += (int64_t)g.mats.size();
        part_off += g.partials_per_mat * (int64_t)g.mats.size();
        P.groups.push_back(std::move(g));
    }
    if (field == Field::MODP) {
        // F_p results are exact whatever the chunking, so a batch too small to
        // fill the GPU gets shorter chunks (down to 2^5 steps, or the whole walk)
        // until the launch holds about 2^18 chunks; pinned lengths are kept.
        const int64_t kTargetItems = (int64_t)1 << 18;
        bool changed = true;
        while (changed) {
            int64_t total = 0;
            for (const auto& g : P.groups) total += g.items;
            if (total >= kTargetItems) break;
            changed = false;
            for (auto& g : P.groups) {
                const int floor_ell = std::min(walk_bits(g.n, g.nw), 5);
                if (tune_get((int)field, g.n) > 0 || g.ell <= floor_ell) continue;
                g.ell -= 1;
                g.log2_chunks += 1;
                g.items <<= 1;
                changed = true;
            }
        }
        part_off = 0;
        for (auto& g : P.groups) {
            const int lg = group_log2(g.log2_chunks, chunks_per_warp(false, false, g.n));
            g.partials_per_mat = (int64_t)1 << (g.log2_chunks - lg);
            g.part_off = part_off;
            part_off += g.partials_per_mat * (int64_t)g.mats.size();
        }
    }
    P.col_elems = col_off;
    P.total_partials = part_off;
    P.batch = batch;
    return P;
}

uint64_t plan_units(const BatchPlan& P) {
    uint64_t u = 0;
    for (auto& g : P.groups) u += (uint64_t)g.mats.size() * (uint64_t)g.n << g.n;
    return u;
}

static int alloc_ws(Workspace& ws, size_t bytes, cudaStream_t s) {
    ws.bytes = bytes;
    if (bytes == 0) return PERMX_OK;
    cudaError_t e = ws_alloc(&ws.base, bytes, s);
    if (e != cudaSuccess) {
        ws.base = nullptr;
        return e == cudaErrorMemoryAllocation ? fail(PERMX_ENOMEM, "workspace allocation failed")
                                              : cuda_fail(e, "workspace allocation");
    }
    return PERMX_OK;
}

// ---------------------------------------------------------------------------
// prepare / execute / release.  prepare() plans the batch, allocates one
// workspace and lays out the metadata (uploaded once, or kept on the host to
// travel as a kernel parameter when it is at most kMetaByValue bytes);
// execute() only enqueues kernels and memsets (so it can be captured in a
// CUDA graph and replayed); release() returns the workspace.  The one-shot
// calls below run all three.
// ---------------------------------------------------------------------------
constexpr size_t kMetaByValue = 16384;

int prepare_batch(Field field, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                  cudaStream_t s, Prepared& X) {
    X = Prepared{};
    X.field = field;
    X.batch = batch;
    X.P = plan_batch(n, batch, field);
    X.x64 = !X.P.groups.empty() && X.P.groups[0].x64;
    const size_t ngroups = X.P.groups.size();
    std::vector<unsigned char> host;
    if (field == Field::MODP) {
        std::vector<StageDesc> stage(batch);
        std::vector<uint32_t> pp(batch), pinv(batch);
        std::vector<ModpFinal> fin(batch);
        for (auto& g : X.P.groups) {
            for (size_t q = 0; q < g.mats.size(); ++q) {
                const int64_t b = g.mats[q], m = g.first_mat + (int64_t)q;
                stage[m] = StageDesc{offset[b], g.col_off + (int64_t)q * g.mat_stride, g.n, g.ld, p[b], g.nw};
                pp[m] = p[b];
                pinv[m] = inv_mod_2_32(p[b]);
                fin[m].p = p[b];
                fin[m].rfix = pow_mod((uint32_t)(((uint64_t)1 << 32) % p[b]), (uint64_t)(g.n - 1), p[b]);
                if (g.nw) fin[m].rfix = (uint32_t)((uint64_t)fin[m].rfix * 2 % p[b]);
                fin[m].negate = g.nw ? !(g.n & 1) : (g.n & 1);
                fin[m].out_index = b;
            }
        }
        X.o_stage = 0;
        X.o_p = align256(X.o_stage + sizeof(StageDesc) * batch);
        X.o_pinv = align256(X.o_p + 4 * batch);
        X.o_fin = align256(X.o_pinv + 4 * batch);
        X.o_meta_end = align256(X.o_fin + sizeof(ModpFinal) * batch);
        X.o_done = X.o_meta_end;
        X.o_acc = align256(X.o_done + 4 * ngroups);
        X.o_zero_end = X.o_acc + 8 * batch;
        X.o_col = align256(X.o_zero_end);
        X.bytes = align256(X.o_col + 4 * (size_t)X.P.col_elems);
        host.resize(X.o_meta_end);
        std::memcpy(host.data() + X.o_stage, stage.data(), sizeof(StageDesc) * batch);
        std::memcpy(host.data() + X.o_p, pp.data(), 4 * batch);
        std::memcpy(host.data() + X.o_pinv, pinv.data(), 4 * batch);
        std::memcpy(host.data() + X.o_fin, fin.data(), sizeof(ModpFinal) * batch);
    } else {
        const bool cplx = field == Field::C128;
        const int w = cplx ? 2 : 1;   // doubles per entry
        std::vector<StageDesc> stage(batch);
        std::vector<FpFinal> fin(batch);
        for (auto& g : X.P.groups) {
            for (size_t q = 0; q < g.mats.size(); ++q) {
                const int64_t b = g.mats[q], m = g.first_mat + (int64_t)q;
                // staging works on entries of w doubles: offsets in entries
                stage[m] = StageDesc{offset[b], (g.col_off / w) + (int64_t)q * (g.mat_stride / w), g.n, g.ld, 0u, g.nw};
                fin[m].first = g.part_off + (int64_t)q * g.partials_per_mat;
                fin[m].count = g.partials_per_mat;
                fin[m].negate = g.nw ? !(g.n & 1) : (g.n & 1);
                fin[m].twice = g.nw;
                fin[m].out_index = b;
            }
        }
        const int pw = fp_slot_doubles(!X.P.groups.empty() && X.P.groups[0].x64, cplx);   // doubles per partial slot
        X.o_stage = 0;
        X.o_fin = align256(sizeof(StageDesc) * batch);
        X.o_meta_end = align256(X.o_fin + sizeof(FpFinal) * batch);
        X.o_done = X.o_meta_end;
        X.o_zero_end = X.o_done + 4 * ngroups;
        X.o_part = align256(X.o_zero_end);
        X.o_col = align256(X.o_part + 8 * (size_t)pw * (size_t)X.P.total_partials);
        X.bytes = align256(X.o_col + 8 * (size_t)X.P.col_elems);
        host.resize(X.o_meta_end);
        std::memcpy(host.data() + X.o_stage, stage.data(), sizeof(StageDesc) * batch);
        std::memcpy(host.data() + X.o_fin, fin.data(), sizeof(FpFinal) * batch);
    }
    Workspace ws;
    int rc = alloc_ws(ws, X.bytes, s);
    if (rc) return rc;
    X.ws = static_cast<unsigned char*>(ws.base);
    if (host.size() <= kMetaByValue) {
        X.meta = std::move(host);   // passed to the set-up kernel of every execution
        return PERMX_OK;
    }
    cudaError_t e = cudaMemcpyAsync(X.ws, host.data(), host.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        release_batch(X, s);
        return cuda_fail(e, "metadata upload");
    }
    return PERMX_OK;
}

void release_batch(Prepared& X, cudaStream_t s) {
    if (X.ws) ws_free(X.ws, s);
    X.ws = nullptr;
}

namespace {

template <int SZ>
cudaError_t launch_setup_sz(const Prepared& X, const void* A, cudaStream_t s) {
    MetaBytes<SZ> m;
    std::memset(&m, 0, sizeof m);
    m.words = (uint32_t)((X.meta.size() + 3) / 4);
    std::memcpy(m.w, X.meta.data(), X.meta.size());
    uint32_t* ws = reinterpret_cast<uint32_t*>(X.ws);
    const uint32_t zf = (uint32_t)(X.o_done / 4), zw = (uint32_t)((X.o_zero_end - X.o_done + 3) / 4);
    const unsigned grid = (unsigned)X.batch;
    if (X.field == Field::MODP) {
        setup_columns_kernel<SZ, uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t*>(A), m, ws, zf, zw,
                                                                reinterpret_cast<uint32_t*>(X.ws + X.o_col));
    } else if (X.x64) {
        int64_t* col = reinterpret_cast<int64_t*>(X.ws + X.o_col);
        if (X.field == Field::C128)
            setup_x64_kernel<SZ, 2><<<grid, kStageX64Threads, 0, s>>>(static_cast<const double*>(A), m, ws, zf, zw, col);
        else
            setup_x64_kernel<SZ, 1><<<grid, kStageX64Threads, 0, s>>>(static_cast<const double*>(A), m, ws, zf, zw, col);
    } else if (X.field == Field::C128) {
        setup_columns_kernel<SZ, double2><<<grid, 256, 0, s>>>(static_cast<const double2*>(A), m, ws, zf, zw,
                                                               reinterpret_cast<double2*>(X.ws + X.o_col));
    } else {
        setup_columns_kernel<SZ, double><<<grid, 256, 0, s>>>(static_cast<const double*>(A), m, ws, zf, zw,
                                                              reinterpret_cast<double*>(X.ws + X.o_col));
    }
    return cudaGetLastError();
}

// Metadata, zeroed words and staging for one execution.
cudaError_t launch_setup(const Prepared& X, const void* A, cudaStream_t s) {
    if (!X.meta.empty()) {
        if (X.meta.size() <= 1024) return launch_setup_sz<1024>(X, A, s);
        if (X.meta.size() <= 4096) return launch_setup_sz<4096>(X, A, s);
        return launch_setup_sz<16384>(X, A, s);
    }
    unsigned char* d = X.ws;
    cudaError_t e = cudaMemsetAsync(d + X.o_done, 0, X.o_zero_end - X.o_done, s);
    if (e != cudaSuccess) return e;
    const StageDesc* sd = reinterpret_cast<const StageDesc*>(d + X.o_stage);
    const unsigned grid = (unsigned)X.batch;
    if (X.field == Field::MODP)
        stage_columns_kernel<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t*>(A), sd,
                                                             reinterpret_cast<uint32_t*>(d + X.o_col));
    else if (X.x64 && X.field == Field::C128)
        stage_x64_kernel<2><<<grid, kStageX64Threads, 0, s>>>(static_cast<const double*>(A), sd,
                                                                reinterpret_cast<int64_t*>(d + X.o_col));
    else if (X.x64)
        stage_x64_kernel<1><<<grid, kStageX64Threads, 0, s>>>(static_cast<const double*>(A), sd,
                                                                reinterpret_cast<int64_t*>(d + X.o_col));
    else if (X.field == Field::C128)
        stage_columns_kernel<double2><<<grid, 256, 0, s>>>(static_cast<const double2*>(A), sd,
                                                            reinterpret_cast<double2*>(d + X.o_col));
    else
        stage_columns_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double*>(A), sd,
                                                           reinterpret_cast<double*>(d + X.o_col));
    return cudaGetLastError();
}

}  // namespace

cudaError_t StreamSet::create(int dev) {
    device = dev;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int q = 0; q < kGroupStreams && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&side[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[q], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) destroy();
    return e;
}

void StreamSet::destroy() {
    for (int q = 0; q < kGroupStreams; ++q) {
        if (side[q]) cudaStreamDestroy(side[q]);
        if (join[q]) cudaEventDestroy(join[q]);
        side[q] = nullptr;
        join[q] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
}

namespace {
// one stream set per device for the lifetime of the calling thread
struct ThreadStreams {
    StreamSet sets[64];
    bool failed[64] = {};
    ~ThreadStreams() {
        for (auto& x : sets)
            if (x.fork) x.destroy();
    }
};
}  // namespace

StreamSet* thread_streams() {
    static thread_local ThreadStreams T;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || T.failed[dev]) return nullptr;
    StreamSet& x = T.sets[dev];
    if (!x.fork && x.create(dev) != cudaSuccess) {
        T.failed[dev] = true;
        cudaGetLastError();
        return nullptr;
    }
    return &x;
}

namespace {

// Launch the walk of every size group, concurrently when there are several:
// each group waits for the staging on `s` (fork event), runs on a stream of
// the set, and `s` waits for all of them before the finalisation (join
// events).  Under stream capture the same calls record a graph with one
// parallel branch per group.
template <typename LaunchGroup>
cudaError_t launch_groups(const Prepared& X, cudaStream_t s, LaunchGroup&& launch) {
    const size_t ng = X.P.groups.size();
    StreamSet* ss = ng > 1 ? (X.streams ? X.streams : thread_streams()) : nullptr;
    if (!ss) {
        for (size_t gi = 0; gi < ng; ++gi) {
            const cudaError_t e = launch(X.P.groups[gi], s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = cudaEventRecord(ss->fork, s);
    const int used = (int)std::min<size_t>(ng, kGroupStreams);
    for (int q = 0; q < used && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(ss->side[q], ss->fork, 0);
    // the largest walk first, so that the smaller groups fill its tail
    std::vector<size_t> order(ng);
    for (size_t gi = 0; gi < ng; ++gi) order[gi] = gi;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const GroupPlan &ga = X.P.groups[a], &gb = X.P.groups[b];
        return (double)ga.mats.size() * ga.n * std::ldexp(1.0, ga.n) >
               (double)gb.mats.size() * gb.n * std::ldexp(1.0, gb.n);
    });
    for (size_t k = 0; k < ng && e == cudaSuccess; ++k) e = launch(X.P.groups[order[k]], ss->side[k % kGroupStreams]);
    // join every stream that waited on the fork, even after a failed launch, so
    // that no side stream is left part of a capture
    for (int q = 0; q < used; ++q) {
        cudaError_t f = cudaEventRecord(ss->join[q], ss->side[q]);
        if (f == cudaSuccess) f = cudaStreamWaitEvent(s, ss->join[q], 0);
        if (e == cudaSuccess) e = f;
    }
    return e;
}

}  // namespace

int execute_batch(const Prepared& X, const void* A, void* out, cudaStream_t s) {
    unsigned char* d = X.ws;
    cudaError_t e = launch_setup(X, A, s);
    const GroupPlan* g0 = X.P.groups.data();
    unsigned* done = reinterpret_cast<unsigned*>(d + X.o_done);
    if (X.field == Field::MODP) {
        const ModpFinal* fin = reinterpret_cast<const ModpFinal*>(d + X.o_fin);
        unsigned long long* acc = reinterpret_cast<unsigned long long*>(d + X.o_acc);
        if (e == cudaSuccess)
            e = launch_groups(X, s, [&](const GroupPlan& g, cudaStream_t ls) {
                ModpLaunch L;
                L.colT = reinterpret_cast<const uint32_t*>(d + X.o_col) + g.col_off;
                L.p = reinterpret_cast<const uint32_t*>(d + X.o_p) + g.first_mat;
                L.pinv = reinterpret_cast<const uint32_t*>(d + X.o_pinv) + g.first_mat;
                L.acc = acc + g.first_mat;
                L.mat_stride = g.mat_stride;
                L.item_begin = 0;
                L.item_end = (uint64_t)g.items;
                L.k_lo = 0;
                L.k_hi = (uint64_t)1 << walk_bits(g.n, g.nw);
                L.ell = g.ell;
                L.log2_chunks = g.log2_chunks;
                L.nw = g.nw;
                const int64_t count = (int64_t)g.mats.size();
                if (count <= kFuseFinalMax) {     // the walk's last block finalises
                    L.fin = fin + g.first_mat;
                    L.nfin = (int)count;
                    L.done = done + (&g - g0);
                    L.out = static_cast<uint32_t*>(out);
                    return dispatch_modp(g.n, L, ls);
                }
                cudaError_t f = dispatch_modp(g.n, L, ls);
                if (f != cudaSuccess) return f;
                finalize_modp_kernel<<<(unsigned)((count + 255) / 256), 256, 0, ls>>>(
                    acc + g.first_mat, fin + g.first_mat, count, static_cast<uint32_t*>(out));
                return cudaGetLastError();
            });
        if (e != cudaSuccess) return cuda_fail(e, "perm_modp launch");
        return PERMX_OK;
    }
    const bool cplx = X.field == Field::C128;
    const int pw = fp_slot_doubles(X.x64, cplx);
    const FpFinal* fin = reinterpret_cast<const FpFinal*>(d + X.o_fin);
    const double* part = reinterpret_cast<const double*>(d + X.o_part);
    if (e == cudaSuccess)
        e = launch_groups(X, s, [&](const GroupPlan& g, cudaStream_t ls) {
            FpLaunch L;
            L.colT = reinterpret_cast<const double*>(d + X.o_col) + g.col_off;
            L.partial = reinterpret_cast<double*>(d + X.o_part) + (size_t)pw * g.part_off;
            L.mat_stride = g.mat_stride;
            L.item_begin = 0;
            L.item_end = (uint64_t)g.items;
            L.ell = g.ell;
            L.log2_chunks = g.log2_chunks;
            L.nw = g.nw;
            const int64_t count = (int64_t)g.mats.size();
            const bool fused = count <= kFuseFinalMax;
            if (fused) {                        // the walk's last block finalises
                L.fin = fin + g.first_mat;
                L.nfin = (int)count;
                L.cplx = cplx ? 1 : 0;
                L.done = done + (&g - g0);
                L.part_all = part;
                L.out = out;
            }
            cudaError_t f;
            if (g.x64) f = cplx ? dispatch_x64c(g.n, L, ls) : dispatch_x64r(g.n, L, ls);
            else f = cplx ? dispatch_c128(g.n, L, ls) : dispatch_f64(g.n, L, ls);
            if (f != cudaSuccess || fused) return f;
            return launch_finalize_fp(part, fin + g.first_mat, count, cplx, g.x64, out, ls);
        });
    if (e != cudaSuccess) return cuda_fail(e, cplx ? "perm_c128 launch" : "perm_f64 launch");
    return PERMX_OK;
}

int run_modp_batch(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                   uint32_t* out, cudaStream_t s) {
    Prepared X;
    int rc = prepare_batch(Field::MODP, n, offset, p, batch, s, X);
    if (rc) return rc;
    rc = execute_batch(X, A, out, s);
    release_batch(X, s);
    return rc;
}

int run_fp_batch(const double* A, const int32_t* n, const int64_t* offset, int64_t batch, void* out, bool cplx,
                 cudaStream_t s) {
    Prepared X;
    int rc = prepare_batch(cplx ? Field::C128 : Field::F64, n, offset, nullptr, batch, s, X);
    if (rc) return rc;
    rc = execute_batch(X, A, out, s);
    release_batch(X, s);
    return rc;
}

}  // namespace permx

namespace permx {
cudaError_t stage_columns_u32(const uint32_t* A, int n, int ld, uint32_t p, int nw, uint32_t* colT,
                              cudaStream_t s) {
    StageDesc h{0, 0, n, ld, p, nw};
    StageDesc* d = nullptr;
    cudaError_t e = ws_alloc(reinterpret_cast<void**>(&d), sizeof h, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        stage_columns_kernel<uint32_t><<<1, 256, 0, s>>>(A, d, colT);
        e = cudaGetLastError();
    }
    cudaError_t f = ws_free(d, s);
    return e != cudaSuccess ? e : f;
}
}  // namespace permx
