/*
 * permx — Gray-code Ryser permanents on one NVIDIA B300 (sm_103a).
 *
 * The operation (paper §1 for the definition and Ryser's O(n 2^n) formula;
 * §2.2 for the Gray-code block evaluation):
 *
 *     perm(A) = sum_{sigma in S_n} prod_i a_{i,sigma(i)}
 *             = (-1)^n  sum_{S subset {0..n-1}} (-1)^{|S|} prod_i sum_{j in S} a_ij .
 *
 * The 2^n subsets are walked in reflected-binary Gray order S_k = k ^ (k>>1):
 * consecutive subsets differ in one column j = ctz(k), so every row sum
 * changes by +-a_ij per step.  Over F_p (paper §2.1) the same sum is taken
 * with residues; for the Schur matrix S_n = (w^{jk}) it is evaluated as the
 * residue matrix (g^{jk} mod p), g a primitive n-th root of unity mod a
 * prime p = 1 (mod n), and the exact integer is recovered by Chinese
 * remaindering over enough primes that prod p > 2 n^{n/2} (|perm(S_n)| <=
 * n^{n/2}, paper §2.1).
 *
 * Conventions for every entry point:
 *  - Return PERMX_OK (0) on success, a negative PERMX_E* code otherwise;
 *    perm_last_error() gives a message for the calling thread's last error.
 *  - Matrices are square, row-major, element (i,j) at A[offset + i*n + j];
 *    complex entries interleave (re, im).
 *  - "device" pointers are CUDA device memory owned by the caller; the library
 *    never frees them.  Host arrays are read before the call returns.
 *  - Asynchronous calls enqueue work on the caller's stream (a cudaStream_t
 *    passed as void*, NULL = the legacy default stream) and return; results
 *    are valid once that stream has been synchronised.  Temporary device
 *    memory is allocated stream-ordered and released on the same stream.
 *  - The library uses whichever CUDA device is current on the calling thread.
 *  - Limits: 1 <= n <= PERMX_MAX_N_FP for float64/complex128 and
 *    1 <= n <= PERMX_MAX_N_MODP for F_p; primes satisfy 2 < p < 2^31.
 */
#ifndef PERMX_H
#define PERMX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PERMX_OK 0
#define PERMX_EINVAL (-1)   /* bad argument: n out of range, NULL pointer, p not an odd prime < 2^31, ... */
#define PERMX_ENOMEM (-2)   /* device or host allocation failed */
#define PERMX_EBUSY (-3)    /* serving: admission is full; retry after polling */
#define PERMX_ECUDA (-4)    /* a CUDA runtime call failed (message has the CUDA error string) */
#define PERMX_ETIMEOUT (-5) /* a bounded wait expired */
#define PERMX_ENOTFOUND (-6) /* serving: unknown ticket */
#define PERMX_EIO (-7)      /* checkpoint file could not be read/written or is corrupt */
#define PERMX_EAGAIN (-8)   /* a long run stopped early at the caller's request; resume from the checkpoint */

#define PERMX_MAX_N_FP 32
#define PERMX_MAX_N_MODP 48

typedef struct { double re, im; } perm_c128_t;

/* Message for the calling thread's most recent failure ("" if none). */
const char* perm_last_error(void);

/* Library version string. */
const char* permx_version(void);

/* ------------------------------------------------------------------------
 * Batched permanents (paper §1 definition, §2.2 Gray-code evaluation; the
 * batches of §3.1, §5.1 and §6 are many independent matrices).
 *
 * A       device, row-major matrices; matrix b starts at element offset[b]
 *         (elements, not bytes) and has n[b]*n[b] entries.
 * n       host array [batch] of sizes.
 * offset  host array [batch] of element offsets into A.
 * batch   number of matrices (0 is allowed and does nothing).
 * out     device array [batch]: out[b] = perm(A_b).
 * stream  cudaStream_t or NULL.
 *
 * Matrices of different sizes may be mixed freely ("ragged").  The work for
 * one matrix is split into Gray-code chunks whose size depends only on
 * (n, field), and the chunk results are combined in a fixed order, so out[b]
 * is bit-for-bit the same whatever else is in the batch.
 * float64 / complex128 arithmetic (permx_set_fp_arith): PERMX_FP_ARITH_INT
 * (default) runs on the integer pipes.  Row i is scaled by a power of two
 * 2^s_i with 2^s_i sum_j |a_ij| in [2^62, 2^63) and its entries rounded to even
 * integers (each entry moves by at most 2^-62 sum_j |a_ij|), so the walk's row
 * sums R of the rounded, scaled matrix are exact int64 values (|R_i| < 2^62 + 2^17);
 * each term multiplies its n row sums with truncated 62-bit integer mantissas
 * (error at most 16n (real) or 64n (complex) times sum_i |R_i|^-1 prod_k |R_k|,
 * a chain's head row sum counting as 2^62 in its first factor; about 2^-58
 * sum_j |a_ij| / |r_i| relative per factor for the unscaled row sum r_i); each
 * chunk adds its terms
 * in 128-bit fixed point (error at most 2^-80 of the sum of the term
 * magnitudes), and the chunk sums are merged in integers (the same 2^-80
 * grid rule) and rounded to float64 once.  The result is not exact: it is
 * perm(A) to within these per-term errors summed over the 2^(n-1) terms, plus
 * the final rounding (measured: 1.7e-15 relative or better against the
 * oracle up to n = 23, on Haar U(23) whose terms cancel by ~1e9).
 * PERMX_FP_ARITH_FP64 uses IEEE float64 row sums and products with TwoSum
 * compensated accumulation.  Both use the Nijenhuis-Wilf form of Ryser's
 * formula (2^(n-1) Gray steps).  A matrix with a NaN or infinite entry gives
 * NaN (NaN + i NaN) in integer mode, without affecting the other matrices;
 * FP64 mode follows IEEE propagation.
 * Errors: PERMX_EINVAL for n[b] outside [1, PERMX_MAX_N_FP], NULL pointers or
 * batch < 0; PERMX_ENOMEM; PERMX_ECUDA.  On error nothing is guaranteed about
 * out.
 * ---------------------------------------------------------------------- */
int perm_c128(const perm_c128_t* A, const int32_t* n, const int64_t* offset, int64_t batch,
              perm_c128_t* out, void* stream);
int perm_f64(const double* A, const int32_t* n, const int64_t* offset, int64_t batch,
             double* out, void* stream);

/* Arithmetic of the float64 / complex128 walks for subsequent calls (process
 * wide): PERMX_FP_ARITH_INT or PERMX_FP_ARITH_FP64 (see above).  Returns the
 * previous mode, or PERMX_EINVAL.  Results differ between the modes only by
 * rounding; within one mode they are bit-reproducible. */
#define PERMX_FP_ARITH_FP64 0
#define PERMX_FP_ARITH_INT 1
int permx_set_fp_arith(int mode);
int permx_get_fp_arith(void);

/* F_p permanents (paper §2.1).  A holds residues mod p[b] (uint32; entries
 * at or above p[b] are taken mod p[b] during staging, so the result is the
 * permanent of A mod p[b]; the checked host path perm_modp_host rejects
 * them instead), p host array [batch] of primes 2 < p < 2^31, out device array
 * [batch] of canonical residues in [0, p[b]).  1 <= n[b] <= PERMX_MAX_N_MODP.
 * Exact: the result does not depend on chunking or batch composition, so a
 * call whose matrices would make fewer than 2^18 chunks shortens its chunks
 * (down to 2^5 Gray steps) to fill the GPU, unless perm_tune_set pinned them. */
int perm_modp(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p,
              int64_t batch, uint32_t* out, void* stream);

/* Host-buffer variants: A and out in host memory; the call copies A to the
 * device, runs the batched path on `stream`, copies out back and
 * synchronises the stream before returning.  The modp variant also checks
 * every entry against its prime (PERMX_EINVAL otherwise). */
int perm_c128_host(const perm_c128_t* A, const int32_t* n, const int64_t* offset, int64_t batch,
                   perm_c128_t* out, void* stream);
int perm_f64_host(const double* A, const int32_t* n, const int64_t* offset, int64_t batch,
                  double* out, void* stream);
int perm_modp_host(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p,
                   int64_t batch, uint32_t* out, void* stream);

/* Permanents of submatrices (paper §8, boson sampling: the amplitude of n
 * photons entering modes c_1..c_n and leaving modes r_1..r_n of an
 * interferometer U is perm(U_T); with repeated modes the probability is
 * |perm(U_T)|^2 / (prod_i s_i! prod_j t_j!), s and t the occupation numbers).
 *   out[b] = perm( U[rows[b*n + i], cols[b*n + j]] )_{i,j < n}
 * U: DEVICE m x m matrix, row-major with row stride ldu >= m entries
 * (complex128: 16-byte aligned).  rows, cols: HOST arrays of batch*n
 * indices in [0, m), repeats allowed; checked before anything is enqueued
 * (EINVAL names the first bad index).  out: DEVICE array of batch values.
 * 1 <= n <= PERMX_MAX_N_FP, m >= 1 (n may exceed m when modes repeat).
 * Asynchronous on `stream` after the host checks, except that copying the
 * index arrays waits for the work already on `stream` (they are copied during
 * the call, so the caller may reuse them at once).  Each result has the bits perm_c128 / perm_f64
 * gives for the extracted n x n matrix.  Errors: EINVAL, ENOMEM, ECUDA. */
int perm_c128_gather(const perm_c128_t* U, int32_t m, int64_t ldu, const int32_t* rows, const int32_t* cols,
                     int32_t n, int64_t batch, perm_c128_t* out, void* stream);
int perm_f64_gather(const double* U, int32_t m, int64_t ldu, const int32_t* rows, const int32_t* cols, int32_t n,
                    int64_t batch, double* out, void* stream);

/* Allocation-free variant of perm_modp (the paper has no counterpart; this is
 * an interface for callers that cannot allocate memory during a call, e.g.
 * because another allocator owns the device memory budget or because the
 * call sits on a latency-critical path that must not enter an allocator).
 * Same arguments, results and exactness as perm_modp, for at most
 * PERMX_NOALLOC_MAX_BATCH matrices per call (any 1 <= n <= 48); larger
 * batches are rejected with PERMX_EINVAL.  It calls no cudaMalloc/cudaFree
 * and allocates no device memory: its intermediates live in one fixed
 * device array of PERMX_NOALLOC_SCRATCH_BYTES bytes that every GPU loading
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls whose GPU work overlaps (other streams or threads on
 * the same device) race and must be serialised by the caller. */
#define PERMX_NOALLOC_MAX_BATCH 64
#define PERMX_NOALLOC_SCRATCH_BYTES (1 << 20)
int perm_modp_noalloc(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p,
                      int64_t batch, uint32_t* out, void* stream);

/* Signed Ryser partial sum of one F_p matrix over a range of Gray indices
 * (paper §2.2: one contiguous Gray-code block):
 *     out = sum_{k0 <= k < k1} (-1)^{|S_k|} prod_i sum_{j in S_k} a_ij  mod p,
 * S_k = k ^ (k >> 1), without the (-1)^n factor.  A is a device n*n matrix,
 * out a host pointer; synchronous.  k0 <= k1 <= 2^n.  Used for checkpointed
 * long runs; summing the ranges of a partition of [0, 2^n) and multiplying
 * by (-1)^n gives perm(A) mod p. */
int perm_modp_gray_range(const uint32_t* A, int32_t n, uint32_t p, uint64_t k0, uint64_t k1,
                         uint32_t* out, void* stream);

/* ------------------------------------------------------------------------
 * Planned batches and CUDA graphs (the batched call of paper §3-§7 repeated
 * over many inputs of one shape).  perm_plan_create fixes field, sizes,
 * offsets and (F_p) primes: it computes the chunk plan, allocates the
 * workspace from the library's pool and uploads the metadata, synchronising
 * `stream`.  perm_plan_execute(A, out) then only enqueues kernels and one
 * memset on `stream` (A, out: device buffers laid out as planned), so it may
 * be captured in a CUDA graph; perm_plan_graph_launch does that capture
 * itself on first use for a given (A, out) pair and afterwards replays the
 * graph with one launch.  The Gray walks of the plan's size groups run
 * concurrently on streams the plan owns (forked from and joined back into
 * `stream`; in a capture, parallel branches of the graph), largest walk
 * first, so small sizes fill the tail of large ones; one-shot batched calls
 * do the same on streams of the calling thread.  Executions of one plan must
 * not overlap on the GPU (they share the workspace).  Errors: EINVAL, ENOMEM,
 * ECUDA.
 * ---------------------------------------------------------------------- */
typedef struct perm_plan perm_plan;
int perm_plan_create(int field, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                     void* stream, perm_plan** plan);
int perm_plan_execute(perm_plan* plan, const void* A, void* out, void* stream);
int perm_plan_graph_launch(perm_plan* plan, const void* A, void* out, void* stream);
int perm_plan_destroy(perm_plan* plan);

/* Several plans (e.g. a complex128 and a float64 batch of paper §3-§7
 * ensembles) captured into ONE CUDA graph: plans[i] runs on A[i] -> out[i]
 * (device buffers laid out as that plan was created), each plan a parallel
 * branch of the graph and each of its size groups a branch of that, so one
 * perm_graph_launch (asynchronous on `stream`) computes every plan's batch
 * with the smaller walks overlapping the larger ones.  Results are
 * bit-identical to perm_plan_execute of each plan.  All plans must belong to
 * the current device, appear once, and not execute elsewhere while a launch
 * of the graph runs (they share their workspaces with it).  count >= 1.
 * perm_graph_create captures on a private stream and synchronises nothing;
 * perm_graph_destroy synchronises the device.  Errors: EINVAL, ECUDA. */
typedef struct perm_graph perm_graph;
int perm_graph_create(perm_plan* const* plans, const void* const* A, void* const* out, int32_t count,
                      perm_graph** graph);
int perm_graph_launch(perm_graph* graph, void* stream);
int perm_graph_destroy(perm_graph* graph);

/* Chunk-length tuning (paper §2.2: the size of a Gray-code block).  The
 * chunk length of a float matrix is 2^ell Gray steps with ell a function of
 * (field, n) only, so float results do not depend on batch composition; they
 * do depend on ell (rounding).  F_p results never depend on ell, and small
 * F_p batches shorten their chunks (see perm_modp).  perm_tune_set
 * pins ell for (field, n) (0 restores the built-in rule; ell <=
 * PERMX_MAX_ELL_MODP for F_p, whose chunk sums of terms below 2^31 are kept
 * in 64 bits and whose walk counts a chunk's steps in 32 bits, ell <=
 * PERMX_MAX_ELL_FP for the float fields, whose exact 128-bit chunk
 * accumulator needs the headroom; EINVAL otherwise); perm_tune_get
 * returns the ell in force; perm_autotune times ell0-3 .. ell0+3 around the
 * built-in rule on a synthetic batch of `batch` n x n matrices (`reps`
 * passes each, each timed on its own; a candidate counts by its fastest pass),
 * keeps the fastest candidate in the table and returns it. */
#define PERMX_MAX_ELL_FP 16
#define PERMX_MAX_ELL_MODP 30
int perm_tune_set(int field, int32_t n, int32_t ell);
int perm_tune_get(int field, int32_t n);
int perm_autotune(int field, int32_t n, int64_t batch, int32_t reps, int32_t* best_ell);
/* Persist the tuning table (host only, no GPU work).  perm_tune_save writes
 * every pinned (field, n, ell) to the text file `path` ("permx-tune 1", then
 * one "field n ell" line per entry) through a temporary file renamed into
 * place; perm_tune_load reads such a file, checks every entry against the
 * perm_tune_set limits and, only if all pass, replaces the whole table
 * (entries absent from the file return to the built-in rule).  Errors:
 * EINVAL (NULL or empty path, malformed, out-of-range or repeated entry,
 * missing header; the table is left unchanged), EIO (the file cannot be
 * opened, read or written). */
int perm_tune_save(const char* path);
int perm_tune_load(const char* path);

/* ------------------------------------------------------------------------
 * Exact perm(S_n) of the Schur matrix S_n = (exp(2 pi i jk/n))_{j,k<n}
 * (paper §1; §2.1 CRT method).
 *
 * n          1 <= n <= PERMX_MAX_N_MODP.
 * nprimes    number of primes; 0 = automatic: ceil(((n/2) log2 n + 2)/30) + 1,
 *            raised if needed until prod p > 2 n^{n/2}.  A request whose
 *            product does not exceed 2 n^{n/2} is rejected (PERMX_EINVAL).
 *            The primes are the largest p < 2^31 with p = 1 (mod n), in
 *            descending order; g is h^((p-1)/n) for the smallest h >= 2 of
 *            order exactly n.  One further prime (the next one below) checks
 *            the reconstruction: its residue must equal the CRT value mod it.
 * ckpt_path  NULL, or a file that records finished primes and the Gray-index
 *            cursor of the current one (written atomically after every slice:
 *            temp file + rename).  An existing, matching file is resumed.
 * out_i128   host [2]: the result as a two's-complement 128-bit integer
 *            (out_i128[0] = low 64 bits, out_i128[1] = high 64 bits); PERMX_EINVAL if it does not fit.
 * out_dec    host buffer for the decimal string (may be NULL).
 * Synchronous.  Errors: PERMX_EINVAL, PERMX_ECUDA, PERMX_EIO, and
 * PERMX_EAGAIN when stopped by perm_schur_crt_ex's slice limit. */
int perm_schur_crt(int32_t n, int32_t nprimes, const char* ckpt_path, int64_t out_i128[2],
                   char* out_dec, size_t out_dec_len);

/* As perm_schur_crt, plus: slice_subsets = Gray indices per device slice
 * between checkpoints (0 = automatic); max_slices = stop with PERMX_EAGAIN
 * after that many slices in this call (0 = no limit); residues_out (host,
 * may be NULL) receives the residue of every prime used, check prime last,
 * and primes_out (host, may be NULL) the primes; both need room for
 * nprimes+1 entries (PERMX_MAX_PRIMES is always enough). */
#define PERMX_MAX_PRIMES 64
int perm_schur_crt_ex(int32_t n, int32_t nprimes, const char* ckpt_path, uint64_t slice_subsets,
                      int64_t max_slices, int64_t out_i128[2], char* out_dec, size_t out_dec_len,
                      uint32_t* residues_out, uint32_t* primes_out);

/* perm(S_n) with the caller's primes: primes[0..count-2] for the CRT and
 * primes[count-1] as the check prime (2 <= count <= PERMX_MAX_PRIMES; each an
 * odd prime below 2^31 with p = 1 (mod n), all distinct, and the product of
 * the first count-1 above 2 n^(n/2); PERMX_EINVAL otherwise, before any GPU
 * work).  For example a second, disjoint prime set cross-checks a long run.
 * Checkpoint, slicing, outputs and errors as perm_schur_crt_ex; residues_out
 * (host, may be NULL) receives count residues. */
int perm_schur_crt_primes(int32_t n, const uint32_t* primes, int32_t count, const char* ckpt_path,
                          uint64_t slice_subsets, int64_t max_slices, int64_t out_i128[2], char* out_dec,
                          size_t out_dec_len, uint32_t* residues_out);

/* One shard of perm(S_n) for a strong split over several GPUs or processes
 * (paper §2.1 CRT method, §2.2 Gray-code blocks: the blocks of every prime
 * are independent, so any set of them can run anywhere and only their sums
 * are exchanged).  The Nijenhuis-Wilf walk of 2^(n-1) Gray indices of every
 * prime primes[i] (i < count) is cut into `slices` equal ranges; work item
 * w = i * slices + j (prime i, range j) belongs to shard w mod nshards.
 * partial_out[i] (host, count entries) receives this shard's signed sum over
 * its ranges of prime i, mod primes[i], without the walk's factor
 * 2 (-1)^(n-1); 0 where the shard has no range of prime i.  Combining: add
 * the shards' partial_out[i] mod primes[i], multiply by 2 (-1)^(n-1) to get
 * perm(S_n) mod primes[i], then reconstruct with perm_crt (use one prime more
 * than the bound needs as a check).  Synchronous, on the current device; the
 * residue matrices are built on the host as in perm_schur_crt.
 * 1 <= n <= PERMX_MAX_N_MODP, 1 <= count <= PERMX_MAX_PRIMES, every prime an
 * odd prime below 2^31 with p = 1 (mod n), slices >= 1, 0 <= shard < nshards.
 * Errors: EINVAL (before any GPU work), ENOMEM, ECUDA. */
int perm_schur_shard(int32_t n, const uint32_t* primes, int32_t count, int32_t slices, int32_t shard,
                     int32_t nshards, uint32_t* partial_out);

/* ------------------------------------------------------------------------
 * Host-side field and CRT helpers (paper §2.1); no GPU needed.
 * ---------------------------------------------------------------------- */
/* The `count` largest primes p < 2^31 with p = 1 (mod n), descending,
 * after skipping the first `skip` of them.  Returns count or a negative code. */
int perm_primes_1_mod_n(int32_t n, int32_t count, int32_t skip, uint32_t* primes_out);
/* g = h^((p-1)/n) for the smallest h >= 2 such that g has order exactly n. */
int perm_primitive_root(uint32_t p, int32_t n, uint32_t* g_out);
/* Residue matrix (g^{jk} mod p), row-major n*n, host memory. */
int perm_schur_residues(int32_t n, uint32_t p, uint32_t g, uint32_t* out);
/* Garner CRT to the symmetric range (-M/2, M/2]; PERMX_EINVAL if the value
 * does not fit in a signed 128-bit integer or k is out of [1, PERMX_MAX_PRIMES]. */
int perm_crt(const uint32_t* residues, const uint32_t* primes, int32_t k, int64_t out_i128[2]);
/* Automatic prime count for perm(S_n) (see perm_schur_crt). */
int perm_schur_prime_count(int32_t n);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of permanent requests (the batches of §3-§7
 * arriving as a stream).  A server owns a CUDA stream, device slots for
 * matrices and partial sums, and a host queue.  serve_submit copies the
 * matrix and returns a ticket at once; admitted requests are advanced by
 * bounded steps (per (field, n) class one wave of Gray-code chunks per step),
 * new arrivals join at the next step, and a request completes when all its
 * chunks are summed.  Each result equals the batched-path result for the same
 * matrix.  Admission takes queued requests in arrival order while three
 * limits allow: the number of resident requests, device memory (a first-fit
 * arena of device_bytes) and outstanding work.  The work of a request is its
 * n 2^(n-1) Gray-walk terms weighted by the cost of its field's term on the
 * GPU (complex128 = 1; float64 = 0.32 and F_p = 0.1 in integer-mantissa mode,
 * complex128 = 3.4 and float64 = 1.4 in FP64 mode), counted until the steps
 * that run its chunks have completed.  A request whose work does not fit lets smaller
 * ones behind it pass, for at most 20 ms; after that nothing passes it until
 * it fits (or nothing else is resident).  Two steps are in flight: the
 * worker plans and enqueues step k+1 while step k runs on the GPU, and reads
 * a step's results once that step has completed.
 * Thread-safe: submit and poll may be called from different threads.
 * ---------------------------------------------------------------------- */
#define PERMX_FIELD_C128 0
#define PERMX_FIELD_F64 1
#define PERMX_FIELD_MODP 2

typedef struct {
    int32_t max_requests;        /* queue + in-flight capacity; submit returns PERMX_EBUSY beyond it (0 = 65536) */
    int32_t max_resident;        /* requests resident on the device at once (0 = 4096) */
    int64_t device_bytes;        /* device memory budget for resident matrices and partials (0 = 1 GiB) */
    int64_t chunks_per_step;     /* Gray-code chunks advanced per step (0 = automatic) */
    int32_t device;              /* CUDA device ordinal */
    int32_t plain_fifo;          /* 1 = baseline: one request at a time, one launch per request */
    int64_t work_budget;         /* outstanding work admitted at once, in complex128-term equivalents
                                    (0 = automatic, 2^35, about 130 ms of the GPU; < 0 = no limit) */
} perm_serve_cfg;

/* Counters of a server (serve_stats2). */
typedef struct {
    int64_t submitted, completed, resident, steps, launches;
    int64_t pending;             /* queued, not yet admitted */
    int64_t resident_work;       /* admitted work not yet run by a completed step (units of work_budget) */
    double gpu_busy_ms;          /* sum over steps of the device time from a step's first to its last operation */
    double uptime_ms;            /* host time since serve_create */
} perm_serve_stats;

typedef struct perm_server perm_server;

int serve_create(const perm_serve_cfg* cfg, perm_server** h);
/* field: PERMX_FIELD_*; A_host: n*n entries (perm_c128_t, double or uint32_t);
 * p: prime for MODP (ignored otherwise).  Errors: EINVAL, EBUSY. */
int serve_submit(perm_server* h, int field, int32_t n, const void* A_host, uint32_t p, uint64_t* ticket);
/* *done = 1 and result written (16, 8 or 4 bytes) when finished, else *done = 0.
 * A finished ticket is released by the poll that reports it. */
int serve_poll(perm_server* h, uint64_t ticket, void* result, int* done);
/* As serve_poll, and on completion also the submit and completion times
 * (nanoseconds on the host's steady clock) measured inside the library. */
int serve_poll_timed(perm_server* h, uint64_t ticket, void* result, int* done, int64_t* t_submit_ns,
                     int64_t* t_done_ns);
/* Block until every submitted request is finished or timeout_ms passes (PERMX_ETIMEOUT). */
int serve_drain(perm_server* h, int64_t timeout_ms);
/* Counters: submitted, completed, resident, steps, launches (host array of 5). */
int serve_stats(perm_server* h, int64_t* stats5);
/* All counters, including the GPU-busy time (gpu_busy_ms / uptime_ms is the
 * fraction of the server's life the GPU spent on its steps). */
int serve_stats2(perm_server* h, perm_serve_stats* out);
int serve_destroy(perm_server* h);

/* ------------------------------------------------------------------------
 * Sample statistics of a batch of permanents, on the device (the
 * distributional measurements of paper §3.2 (Haar unitary: E|perm|^2,
 * circularity), §5.1 Table "orthogonal" (variance and excess kurtosis of
 * perm(O)), §6.1 (real-valuedness of Hermitian permanents), §7.2 Table
 * "lognormal" (skewness and excess kurtosis of log|perm|) and the
 * anti-concentration probabilities Pr[|perm|^2 >= threshold]).
 *
 * values: `count` device values, complex128 (field PERMX_FIELD_C128,
 * 16-byte aligned) or float64 (PERMX_FIELD_F64, imaginary part 0).
 * out: ONE perm_stats_t in DEVICE memory (8-byte aligned), written by the
 * last kernel; ready after `stream` is synchronised.  Moments are the
 * plain (biased, divide by count) sample moments; central moments come from
 * a second pass about the first pass's means.  With |z|^2 := rn(rn(re*re) +
 * rn(im*im)) and |z| := sqrt(|z|^2) (correctly rounded, no fused multiply-
 * add):
 *   count_nonzero  samples with |z|^2 > 0 (the log moments use only these,
 *                  with log|z| := log(|z|^2) / 2; NaN when there are none)
 *   count_above    samples with |z|^2 >= threshold
 *   count_real     samples with |Im z| <= real_tol * |z| (every sample of a
 *                  float64 input)
 * skew = m3 / m2^1.5 and excess kurtosis = m4 / m2^2 - 3 (NaN when m2 = 0).
 * Deterministic: the reduction order depends on count only.  Errors: EINVAL
 * (field MODP, count < 1, NULL or misaligned pointer, real_tol < 0 or NaN),
 * ENOMEM, ECUDA.  Workspace comes from the library pool (stream-ordered). */
typedef struct {
    int64_t count, count_nonzero, count_above, count_real;
    double mean_re, mean_im;
    double var_re, var_im, cov_re_im;   /* central second moments */
    double skew_re, exkurt_re;          /* of Re z */
    double mean_abs2, mean_abs4;        /* E|z|^2, E|z|^4 */
    double mean_z2_re, mean_z2_im;      /* E[z^2] (pseudo-covariance about 0) */
    double min_abs2, max_abs2;
    double log_mean, log_var, log_skew, log_exkurt;   /* of log|z| over nonzero samples */
} perm_stats_t;
int perm_sample_stats(int field, const void* values, int64_t count, double threshold, double real_tol,
                      perm_stats_t* out, void* stream);

/* Histogram of |z|^2 (PERMX_HIST_ABS2, formed as in perm_sample_stats), Re z
 * (PERMX_HIST_RE) or Im z (PERMX_HIST_IM) over the `count` device values:
 * the binned distributions behind the paper's distribution comparisons (§3.2:
 * |perm U|^2 of Haar unitaries against the exponential law; §5-§7: the
 * ensembles' Q-Q plots and tail probabilities).  Inputs and outputs:
 * edges = HOST array of nedges strictly increasing doubles (1..4097);
 * counts = DEVICE int64 array of nedges + 1, overwritten: counts[0] values
 * below edges[0], counts[b] values in [edges[b-1], edges[b]), counts[nedges]
 * values at or above edges[nedges-1]; a value whose selected quantity is NaN
 * is not counted (NaN + 0i counts in the Im histogram as 0).  A value
 * equal to an edge goes to the bin that edge opens.  Edges spaced in
 * geometric progression on |z|^2 bin log|z| without taking a logarithm.
 * Asynchronous on `stream` (the edges are copied during the call).
 * Errors: EINVAL (field MODP, bad kind, NULL or misaligned pointer, bad
 * edges, count < 0), ENOMEM, ECUDA. */
#define PERMX_HIST_ABS2 0
#define PERMX_HIST_RE 1
#define PERMX_HIST_IM 2
int perm_sample_histogram(int field, const void* values, int64_t count, int kind, const double* edges,
                          int32_t nedges, int64_t* counts, void* stream);

/* Measurement hook (the paper has no counterpart): issue-rate probe of one
 * operation kind, the denominator of the walks' pipe rooflines.  Runs
 * `blocks` x `threads` threads (threads in [32, 1024]), each with 8
 * independent chains of `iters` operations, on the current device and
 * stream 0 (synchronous); *ops_per_s = blocks*threads*iters*8 / time,
 * *ms_out (may be NULL) = the CUDA-event time of the timed launch.  Kinds:
 *   0 fma.rn.f64   1 add.rn.f64   2 mul.rn.f64   3 fma.rn.f32
 *   4 mad.lo.u32   5 mul.wide.u32 6 mul.hi.u32   7 add.u32   8 min.u32
 *   9 one F_p term (modular add + Montgomery product)
 *  10 one float64 term in FP64 (add + multiply)
 *  11 one complex128 term in FP64 (2 adds + complex multiply)
 *  12 clz.b64   13 clz.b32
 *  14 one real integer-mantissa combining factor (m m' >> 62)
 *  15 one complex integer-mantissa combining factor
 *  16 one real integer-mantissa term (int64 row-sum update + chain factor m R >> 64)
 *  17 one complex integer-mantissa term (two int64 updates + complex chain factor)
 * Errors: EINVAL (bad kind or sizes, NULL ops_per_s), ENOMEM, ECUDA. */
int permx_peak_probe(int kind, int blocks, int threads, int iters, double* ops_per_s, double* ms_out);

#ifdef __cplusplus
}
#endif
#endif /* PERMX_H */
