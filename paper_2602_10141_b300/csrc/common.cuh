// Internal definitions shared by the permx CUDA sources (not a public header).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <string>

#include "permx.h"

namespace permx {

// ---------------------------------------------------------------------------
// error reporting (thread-local last error, see perm_last_error)
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PERMX_CUDA(call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Chunk plan (paper §2.2: contiguous Gray-code blocks).  A chunk is L = 2^ell
// consecutive Gray indices of a walk over `bits` subset bits (n for plain
// Ryser, n - 1 for the Nijenhuis-Wilf form below).  ell depends only on
// (n, field, form), so a matrix is always cut the same way, whatever batch it
// is in.
//
// Nijenhuis-Wilf form of Ryser's formula ("nw"): with
//     x_i = a_{i,n-1} - (1/2) sum_j a_ij,
//     perm(A) = (-1)^{n-1} 2 sum_{S subset {0..n-2}} (-1)^{|S|} prod_i (x_i + sum_{j in S} a_ij),
// i.e. half the subsets of plain Ryser at the same cost per subset.  The
// staged matrix then carries x as an extra column (index n).
// ---------------------------------------------------------------------------
int chunk_log2_modp(int bits);
// longest F_p chunk (log2 steps): the walk counts k mod 2^(ell+1) in 32 bits
constexpr int kModpMaxEll = PERMX_MAX_ELL_MODP;
static_assert(kModpMaxEll <= 30, "32-bit step counter");
int chunk_log2_fp(int bits);
inline int walk_bits(int n, int nw) { return nw ? n - 1 : n; }

// Padded column length: columns start on 16-byte boundaries.
__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }
__host__ __device__ constexpr int pad2(int n) { return (n + 1) & ~1; }

// ---------------------------------------------------------------------------
// Launch descriptors.  One launch covers a group of matrices that share n.
// Batch mode (segs == nullptr): work item i (item_begin <= i < item_end) is
// chunk (i & (chunks-1)) of matrix (i >> log2_chunks) of the group.
// Segment mode (serving): item i belongs to the last segment s with
// segs[s].item_start <= i and is chunk segs[s].chunk0 + (i - item_start) of
// that segment's matrix, if below segs[s].chunk_end.  Segment starts are
// aligned to min(chunks, 32) items so that a lane group never spans two
// matrices and always holds the same chunks as in batch mode.
// ---------------------------------------------------------------------------
struct SegDesc {
    int64_t item_start;            // first launch item of the segment
    uint64_t chunk0, chunk_end;    // chunk range of the matrix advanced by this segment
    int64_t col_off;               // staged columns at colT + col_off
    int64_t out_off;               // modp: accumulator acc[out_off]; fp: partial slot of chunk 0
    uint32_t p, pinv;              // modp only
};

#ifdef __CUDACC__
__device__ __forceinline__ int find_segment(const SegDesc* __restrict__ segs, int nsegs, uint64_t item) {
    int lo = 0, hi = nsegs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint64_t)__ldg(reinterpret_cast<const long long*>(&segs[mid].item_start)) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#endif

// Finalisation of one matrix (the fixed-order sum of its chunk partials).
struct ModpFinal {
    uint32_t p, rfix;       // rfix = 2^(32(n-1)) mod p undoes the Montgomery factors (times 2 in NW form)
    int32_t negate;         // (-1)^n
    int32_t pad_;
    int64_t out_index;
};
// Integer-mode partial of one chunk lane group and component: the group's
// exact 128-bit fixed-point sum (hi:lo) * 2^e, the matrix's staging scale
// included in e.  flag: 0 no term, 1 a sum, 2 the matrix has a non-finite
// entry.  The finalisation merges these in integers and rounds once.
struct alignas(16) XPart {
    uint64_t lo;
    int64_t hi;
    int32_t e;
    int32_t flag;
    int64_t pad;
};
// doubles per partial slot: FP64 mode (sum, compensation) per component,
// integer mode one XPart per component
constexpr int fp_slot_doubles(bool x64, bool cplx) { return x64 ? (cplx ? 8 : 4) : (cplx ? 4 : 2); }

struct FpFinal {
    int64_t first, count;   // partial slots of this matrix
    int64_t out_index;
    int32_t negate;         // multiply by -1
    int32_t twice;          // multiply by 2 (Nijenhuis-Wilf form)
};

// A walk launch of a group of at most kFuseFinalMax matrices finalises them in
// its last block (the block that takes the last ticket of `done`), which
// saves the finalisation launch of a lone matrix; the arithmetic is the
// finalize kernels' own, so the bits are the same either way.
constexpr int kFuseFinalMax = 4;

struct ModpLaunch {
    const uint32_t* colT;          // group columns: matrix m at colT + m*mat_stride, column j at + j*pad4(n)
    const uint32_t* p;             // per-matrix prime
    const uint32_t* pinv;          // per-matrix p^{-1} mod 2^32
    unsigned long long* acc;       // per-matrix accumulator (sum of partials, each < p)
    int64_t mat_stride;            // elements between matrices
    uint64_t item_begin, item_end; // item range of this launch
    uint64_t k_lo, k_hi;           // Gray-index window applied to every chunk (0, 2^n for a full permanent)
    int ell;                       // log2 chunk length
    int log2_chunks;               // log2 chunks per matrix (walk bits - ell)
    const SegDesc* segs = nullptr; // segment mode when non-null
    int nsegs = 0;
    int nw = 0;                    // 1: Nijenhuis-Wilf form (x column at index n)
    // fused finalisation (batch mode, small groups): matrix m of the group has
    // accumulator acc[m] and descriptor fin[m]; nullptr = a separate kernel
    const ModpFinal* fin = nullptr;
    int nfin = 0;
    unsigned* done = nullptr;      // ticket counter, 0 before the launch, reset to 0 by the last block
    uint32_t* out = nullptr;
    uint32_t zero = 0;             // always 0: keeps the F_p walk's adds on the ALU pipe (ryser_modp.cuh)
};

struct FpLaunch {
    const double* colT;            // group columns (complex: interleaved), matrix m at colT + m*mat_stride
    double* partial;               // per item: (s, c) for real, (s_re, c_re, s_im, c_im) for complex
    int64_t mat_stride;            // doubles between matrices
    uint64_t item_begin, item_end;
    int ell;
    int log2_chunks;
    const SegDesc* segs = nullptr; // segment mode when non-null
    int nsegs = 0;
    int nw = 0;                    // 1: Nijenhuis-Wilf form (x column at index n)
    // fused finalisation (batch mode, small groups): descriptors fin[0..nfin)
    // index the whole batch's partial slots at part_all; nullptr = a separate kernel
    const FpFinal* fin = nullptr;
    int nfin = 0;
    int cplx = 0;
    unsigned* done = nullptr;      // ticket counter, 0 before the launch, reset to 0 by the last block
    const double* part_all = nullptr;
    void* out = nullptr;
};

template <int N> cudaError_t launch_modp(const ModpLaunch& L, int grid, int threads, cudaStream_t s);
template <int N> cudaError_t launch_f64(const FpLaunch& L, int grid, int threads, cudaStream_t s);
template <int N> cudaError_t launch_c128(const FpLaunch& L, int grid, int threads, cudaStream_t s);
template <int N> cudaError_t launch_x64r(const FpLaunch& L, int grid, int threads, cudaStream_t s);
template <int N> cudaError_t launch_x64c(const FpLaunch& L, int grid, int threads, cudaStream_t s);
template <int N> int blocks_per_sm_x64r();
template <int N> int blocks_per_sm_x64c();
template <int N> int blocks_per_sm_modp();
template <int N> int blocks_per_sm_f64();
template <int N> int blocks_per_sm_c128();

// dispatch on runtime n (defined in dispatch.cu)
cudaError_t dispatch_modp(int n, const ModpLaunch& L, cudaStream_t s);
cudaError_t dispatch_f64(int n, const FpLaunch& L, cudaStream_t s);
cudaError_t dispatch_c128(int n, const FpLaunch& L, cudaStream_t s);
cudaError_t dispatch_x64r(int n, const FpLaunch& L, cudaStream_t s);
cudaError_t dispatch_x64c(int n, const FpLaunch& L, cudaStream_t s);
int dispatch_blocks_per_sm(int kind, int n);

// Complex integer-mantissa walks with n > 16 run two lanes per chunk, so a
// warp covers 16 chunks instead of 32; chunk lane groups (and the partial
// slots per matrix) follow from this.
#ifndef PERMX_X64C_PAIR_MIN_N
#define PERMX_X64C_PAIR_MIN_N 17   // complex integer-mantissa walks with n >= this use two lanes per chunk
#endif
// (pairing from n = 10 measured 15 % faster for one lone matrix at n = 14-16 but
// 20 % slower for batches of thousands, which is what the threshold serves)
static_assert(PERMX_X64C_PAIR_MIN_N >= 8, "each lane of a pair needs at least four rows");
constexpr bool x64c_paired(int n) { return n >= PERMX_X64C_PAIR_MIN_N; }
inline int chunks_per_warp(bool x64, bool cplx, int n) { return (x64 && cplx && x64c_paired(n)) ? 16 : 32; }
inline int group_log2(int log2_chunks, int per_warp) {
    const int w = per_warp == 16 ? 4 : 5;
    return log2_chunks < w ? log2_chunks : w;
}   // kind: 0 modp, 1 f64, 2 c128, 3 x64 real, 4 x64 complex

// Arithmetic of the float64 / complex128 walks: 0 = the FP64 pipe (IEEE
// float64 row sums and products), 1 = integer mantissas (exact fixed-point
// row sums, 62-bit products); see include/permx.h, permx_set_fp_arith.
int fp_arith();

constexpr int kRyserThreads = 256;

// Resident blocks per SM of a walk kernel at kRyserThreads threads, queried
// once per kernel.  The cache is atomic because the server's worker thread
// and the caller's threads may make the first call at the same time.
template <typename K>
int occupancy_blocks(std::atomic<int>& slot, K kernel) {
    int b = slot.load(std::memory_order_relaxed);
    if (b > 0) return b;
    b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kRyserThreads, 0) != cudaSuccess || b < 1) b = 1;
    slot.store(b, std::memory_order_relaxed);
    return b;
}

int sm_count();
cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s);   // library memory pool, stream-ordered
cudaError_t ws_free(void* p, cudaStream_t s);

// host helpers (field.cpp)
bool is_prime_u32(uint32_t p);
uint32_t inv_mod_2_32(uint32_t p);                  // p odd: p * inv = 1 (mod 2^32)
uint32_t pow_mod(uint32_t b, uint64_t e, uint32_t p);

}  // namespace permx
