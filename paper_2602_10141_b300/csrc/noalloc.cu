// perm_modp_noalloc: the batched F_p permanent without any memory allocation.
//
// Some callers cannot allocate memory at call time: code that runs while
// another component owns the whole device memory budget (a caching allocator
// that has reserved it, a serving process with a fixed memory plan), real-time
// or latency-critical paths that must not hit the allocator or its
// synchronisation, and embedders whose policy forbids library-side
// allocation.  For them this entry point runs the same staging, Gray-code
// walk and finalisation as perm_modp, but every intermediate (the column-major
// copies, the per-matrix primes and Montgomery constants, the accumulators)
// lives in one fixed array in device global memory, defined below.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it (PERMX_NOALLOC_SCRATCH_BYTES) until the process exits.  In
// host code its name only stands for a host-side shadow symbol, not a device
// address; the device address is obtained with cudaGetSymbolAddress once per
// device, by the first call made on that device, with that device current.
// That first call should therefore come before any stream capture begins.
// All calls share the array and it keeps the last call's contents; each call
// clears what must start at zero (the accumulators).  Calls whose work
// overlaps on the GPU (different streams, or different host threads on one
// device) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "permx.h"

namespace permx {
namespace {

// Fixed scratch for every call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PERMX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxB = PERMX_NOALLOC_MAX_BATCH;

// Everything the set-up kernel needs, passed by value as a kernel parameter
// (no device-side metadata buffer, so no copy and no allocation).
struct NoallocArgs {
    int32_t count;
    int32_t n[kMaxB];              // plan order (sorted by n)
    int64_t src[kMaxB];            // element offset of the matrix in A
    int64_t col[kMaxB];            // word offset of its staged columns in the scratch
    uint32_t p[kMaxB], pinv[kMaxB], rfix[kMaxB];
    int64_t out_index[kMaxB];      // position in the caller's output array
};

// scratch layout: [p: kMaxB u32][pinv: kMaxB u32][acc: kMaxB u64][columns ...]
constexpr size_t kOffP = 0;
constexpr size_t kOffPinv = kOffP + 4 * kMaxB;
constexpr size_t kOffAcc = kOffPinv + 4 * kMaxB;
constexpr size_t kOffCol = ((kOffAcc + 8 * kMaxB) + 255) & ~size_t(255);
static_assert(kOffCol < PERMX_NOALLOC_SCRATCH_BYTES, "scratch layout");

// One block per matrix: primes and constants into the scratch, the
// accumulator cleared, the matrix copied column-major with zero padding.
__global__ void noalloc_setup_kernel(const uint32_t* __restrict__ A, const NoallocArgs args,
                                     unsigned char* __restrict__ scratch) {
    const int k = blockIdx.x;
    const int n = args.n[k], ld = pad4(n);
    uint32_t* colT = reinterpret_cast<uint32_t*>(scratch + kOffCol) + args.col[k];
    if (threadIdx.x == 0) {
        reinterpret_cast<uint32_t*>(scratch + kOffP)[k] = args.p[k];
        reinterpret_cast<uint32_t*>(scratch + kOffPinv)[k] = args.pinv[k];
        reinterpret_cast<unsigned long long*>(scratch + kOffAcc)[k] = 0ull;
    }
    // Nijenhuis-Wilf column x_i = a_{i,n-1} - (1/2) sum_j a_ij mod p, with 1/2 = (p+1)/2
    const uint64_t p = args.p[k];
    for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
        const int j = e / ld, i = e % ld;
        const uint32_t a = i < n ? A[args.src[k] + (int64_t)i * n + j] : 0u;
        colT[e] = a < p ? a : (uint32_t)(a % p);   // residues at or above p taken mod p
    }
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
        uint32_t x = 0;
        if (i < n) {
            const uint32_t* row = A + args.src[k] + (int64_t)i * n;
            uint64_t sum = 0;
            for (int j = 0; j < n; ++j) sum += row[j];
            const uint64_t half = (sum % p) * ((p + 1) / 2) % p;
            x = (uint32_t)(((uint64_t)row[n - 1] + p - half) % p);
        }
        colT[(int64_t)n * ld + i] = x;
    }
}

__global__ void noalloc_finalize_kernel(const NoallocArgs args, const unsigned char* __restrict__ scratch,
                                        uint32_t* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= args.count) return;
    const uint64_t p = args.p[k];
    const unsigned long long acc = reinterpret_cast<const unsigned long long*>(scratch + kOffAcc)[k];
    // rfix = 2 R^(n-1) mod p; perm = (-1)^(n-1) 2 sum
    uint32_t v = (uint32_t)((acc % p) * (uint64_t)args.rfix[k] % p);
    if (!(args.n[k] & 1) && v) v = (uint32_t)p - v;
    out[args.out_index[k]] = v;
}

// device address of the scratch, looked up once per device
std::mutex g_addr_mu;
unsigned char* g_addr[64] = {nullptr};

int scratch_address(unsigned char** out) {
    int dev = 0;
    PERMX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PERMX_EINVAL, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                       "cudaGetSymbolAddress(noalloc scratch)");
        g_addr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_addr[dev];
    return PERMX_OK;
}

}  // namespace
}  // namespace permx

using namespace permx;

extern "C" int perm_modp_noalloc(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p,
                                 int64_t batch, uint32_t* out, void* stream) {
    clear_error();
    if (batch < 0) return fail(PERMX_EINVAL, "batch < 0");
    if (batch == 0) return PERMX_OK;
    if (batch > kMaxB)
        return fail(PERMX_EINVAL, "perm_modp_noalloc: batch exceeds PERMX_NOALLOC_MAX_BATCH (64) matrices per call");
    if (!A || !n || !offset || !p || !out) return fail(PERMX_EINVAL, "NULL pointer argument");

    // plan on the stack: matrices sorted by n (insertion sort, stable)
    int order[kMaxB];
    for (int b = 0; b < (int)batch; ++b) {
        if (n[b] < 1 || n[b] > PERMX_MAX_N_MODP) return fail(PERMX_EINVAL, "n out of range [1, 48]");
        if (offset[b] < 0) return fail(PERMX_EINVAL, "negative offset");
        if (p[b] <= 2 || p[b] >= (1u << 31) || !is_prime_u32(p[b]))
            return fail(PERMX_EINVAL, "p is not an odd prime below 2^31");
        int k = b;
        while (k > 0 && n[order[k - 1]] > n[b]) {
            order[k] = order[k - 1];
            --k;
        }
        order[k] = b;
    }
    static NoallocArgs args;   // host-side argument block (not heap; reused under the lock below)
    static std::mutex args_mu;
    std::lock_guard<std::mutex> lk(args_mu);
    args.count = (int32_t)batch;
    size_t words = 0;
    for (int k = 0; k < (int)batch; ++k) {
        const int b = order[k];
        args.n[k] = n[b];
        args.src[k] = offset[b];
        args.col[k] = (int64_t)words;
        args.p[k] = p[b];
        args.pinv[k] = inv_mod_2_32(p[b]);
        args.rfix[k] = (uint32_t)((uint64_t)pow_mod((uint32_t)((1ull << 32) % p[b]), (uint64_t)(n[b] - 1), p[b]) *
                                  2 % p[b]);
        args.out_index[k] = b;
        words += (size_t)(n[b] + 1) * pad4(n[b]);   // n columns and the x column
    }
    if (kOffCol + 4 * words > (size_t)PERMX_NOALLOC_SCRATCH_BYTES)
        return fail(PERMX_EINVAL, "perm_modp_noalloc: matrices exceed PERMX_NOALLOC_SCRATCH_BYTES");

    unsigned char* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_setup_kernel<<<(unsigned)batch, 256, 0, s>>>(A, args, scratch);
    PERMX_CUDA(cudaGetLastError());
    // one Ryser launch per run of equal n
    for (int k0 = 0; k0 < (int)batch;) {
        int k1 = k0;
        while (k1 < (int)batch && args.n[k1] == args.n[k0]) ++k1;
        const int nn = args.n[k0];
        ModpLaunch L;
        L.colT = reinterpret_cast<const uint32_t*>(scratch + kOffCol) + args.col[k0];
        L.p = reinterpret_cast<const uint32_t*>(scratch + kOffP) + k0;
        L.pinv = reinterpret_cast<const uint32_t*>(scratch + kOffPinv) + k0;
        L.acc = reinterpret_cast<unsigned long long*>(scratch + kOffAcc) + k0;
        L.mat_stride = (int64_t)(nn + 1) * pad4(nn);
        const int bits = walk_bits(nn, 1);   // Nijenhuis-Wilf form: 2^(nn-1) Gray steps
        L.ell = chunk_log2_modp(bits);
        // exact arithmetic: shorter chunks when the run is too small to fill the GPU
        while (L.ell > (bits < 5 ? bits : 5) && ((int64_t)(k1 - k0) << (bits - L.ell)) < ((int64_t)1 << 18)) --L.ell;
        L.log2_chunks = bits - L.ell;
        L.item_begin = 0;
        L.item_end = (uint64_t)(k1 - k0) << L.log2_chunks;
        L.k_lo = 0;
        L.k_hi = 1ull << bits;
        L.nw = 1;
        PERMX_CUDA(dispatch_modp(nn, L, s));
        k0 = k1;
    }
    noalloc_finalize_kernel<<<(unsigned)((batch + 127) / 128), 128, 0, s>>>(args, scratch, out);
    PERMX_CUDA(cudaGetLastError());
    return PERMX_OK;
}
