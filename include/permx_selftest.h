/*
 * Self-test hooks: the integer-mantissa arithmetic of permx's float64 /
 * complex128 walks (the paper has no counterpart; they check this library's
 * own number format) and the batched path's chunk plan.  They run the same
 * host+device helper functions and the same planner the GPU path uses, on
 * the CPU, so both can be checked without a GPU (the arithmetic against exact
 * big-integer results).  They compute no permanents.
 */
#ifndef PERMX_SELFTEST_H
#define PERMX_SELFTEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* (a * b) >> 62, truncated, for |a|, |b| <= 2^62: the kernels' 64x64 product. */
int64_t permx_x64_mulhi62(int64_t a, int64_t b);

/* (a * b) >> 64, truncated, for |a| <= 2^62 + 2^32, |b| < 2^63 - 2^32: the
 * walks' chain factor (a mantissa times a staged row sum). */
int64_t permx_x64_mulhi64(int64_t a, int64_t b);

/* Both products above as the GPU computes them, for count (1..2^20) pairs of
 * HOST arrays a, b; results to HOST arrays hi62, hi64.  Synchronous, on the
 * current device; the caller checks them against the host forms.  Errors:
 * PERMX_EINVAL (NULL pointer, count out of range), PERMX_ENOMEM, PERMX_ECUDA. */
int permx_x64_mulhi_device(const int64_t* a, const int64_t* b, int64_t count, int64_t* hi62, int64_t* hi64);

/* Complex product (ar + i ai)(br + i bi) >> sh by components (sh = 64: the
 * walks' chain factor; sh = 62: the combining factor), for
 * |ar| + |ai|, |br| + |bi| <= 2^62 + 2^20: Karatsuba on the truncated products
 * above, each component within 4 of the exact value.  Returns PERMX_EINVAL for
 * another sh or a NULL output. */
int permx_x64c_mulhi(int64_t ar, int64_t ai, int64_t br, int64_t bi, int32_t sh, int64_t* re, int64_t* im);

/* The same on the GPU for count (1..2^20) HOST 4-tuples in4 = (ar, ai, br, bi):
 * out4 (HOST) = (re, im) for sh = 64, then (re, im) for sh = 62.  Synchronous.
 * Errors: PERMX_EINVAL, PERMX_ENOMEM, PERMX_ECUDA. */
int permx_x64c_mulhi_device(const int64_t* in4, int64_t count, int64_t* out4);

/* The double nearest to (hi 2^64 + lo) 2^e, ties to even (hi:lo a signed
 * 128-bit integer), computed in integer operations as the integer-mode
 * finalisation rounds a matrix's exact fixed-point sum once; subnormal results
 * are rounded at their own precision, too large ones give +-inf. */
double permx_x64_to_double(int64_t hi, uint64_t lo, int32_t e);

/* round(a 2^k) to the nearest integer, ties to even, as staging converts a
 * float entry to the integer-mantissa walk's format (finite a, |a 2^k| < 2^62). */
int64_t permx_x64_scaled_round(double a, int32_t k);

/* Product of n exact integer row sums R[0..n) (|R| < 2^62 + 2^17) as the real walk
 * forms it (four interleaved chains, then combined): value m * 2^e. */
int permx_x64_product(const int64_t* R, int32_t n, int64_t* m_out, int32_t* e_out);

/* Complex version: rows (Rr[i] + i Ri[i]), |Rr[i]| + |Ri[i]| < 2^62 + 2^17;
 * value (re + i im) * 2^e. */
int permx_x64c_product(const int64_t* Rr, const int64_t* Ri, int32_t n, int64_t* re_out, int64_t* im_out,
                       int32_t* e_out);

/* Chunk accumulator: sum_k (-1)^neg[k] m[k] 2^e[k] for k < count (count <= 4096),
 * returned as the double-double hi + lo scaled by 2^scale. */
int permx_x64_accumulate(const int64_t* m, const int32_t* e, const int32_t* neg, int32_t count, int32_t scale,
                         double* hi, double* lo);

/* The same sum split into `parts` consecutive runs (parts a power of two,
 * <= 32), one accumulator per run, merged as the kernels merge the lanes of
 * a group (xor butterfly of symmetric merges), then returned as above.  With
 * swap != 0 every merge takes its operands in the other order; the bits must
 * not change. */
int permx_x64_accumulate_merged(const int64_t* m, const int32_t* e, const int32_t* neg, int32_t count,
                                int32_t parts, int32_t swap, int32_t scale, double* hi, double* lo);

/* The batched path's chunk plan (paper §2.2 Gray-code blocks) for `batch`
 * matrices of sizes n[0..batch) in field `field` (PERMX_FIELD_*), computed on
 * the host exactly as perm_c128 / perm_f64 / perm_modp compute it, with no
 * GPU work.  One row of PERMX_PLAN_COLS int64 per group of equal n, in plan
 * order: n, ell (log2 Gray steps per chunk), log2_chunks (per matrix), ld
 * (padded column length), mat_stride (staged elements per matrix), col_off
 * (first staged element of the group), items (chunks in the group),
 * partials_per_mat, part_off (first partial slot), x64 (1: integer-mantissa
 * walk), nmats.  order (host, batch entries) receives the batch indices in
 * plan order; totals[0] = staged elements, totals[1] = partial slots.
 * Returns the number of groups, or PERMX_EINVAL (bad field, n or pointer,
 * more groups than max_groups). */
#define PERMX_PLAN_COLS 11

/* The serving arena (admission by device memory, serve_*) on its own, on the
 * host: an arena of `capacity` bytes runs `nops` operations ops[2k], ops[2k+1]:
 * (0, bytes) allocates and records results[3k] = offset or -1; (1, j)
 * releases the block allocated by operation j (which must have succeeded and
 * not been released).  After each operation results[3k+1] = bytes in use and
 * results[3k+2] = the largest free block.  Returns the number of free blocks
 * at the end, or PERMX_EINVAL for a bad operation. */
int permx_arena_run(int64_t capacity, const int64_t* ops, int32_t nops, int64_t* results);
int permx_plan_describe(int field, const int32_t* n, int64_t batch, int64_t* groups, int32_t max_groups,
                        int64_t* order, int64_t* totals);

#ifdef __cplusplus
}
#endif
#endif /* PERMX_SELFTEST_H */
