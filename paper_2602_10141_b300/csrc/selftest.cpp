// CPU entry points for the integer-mantissa helpers (include/permx_selftest.h).
// They call the very functions the float64 / complex128 kernels inline.
#include "permx_selftest.h"

#include <vector>

#include "arena.h"
#include "batch.h"
#include "common.cuh"
#include "permx.h"
#include "x64_arith.cuh"

using namespace permx;

extern "C" {

int64_t permx_x64_mulhi62(int64_t a, int64_t b) { return x64_mulhi62(a, b); }

int64_t permx_x64_mulhi64(int64_t a, int64_t b) { return x64_mulhi64(a, b); }

int permx_x64c_mulhi(int64_t ar, int64_t ai, int64_t br, int64_t bi, int32_t sh, int64_t* re, int64_t* im) {
    if (!re || !im || (sh != 62 && sh != 64)) return PERMX_EINVAL;
    if (sh == 64) x64c_mulhi<64>(ar, ai, br, bi, *re, *im);
    else x64c_mulhi<62>(ar, ai, br, bi, *re, *im);
    return PERMX_OK;
}

int64_t permx_x64_scaled_round(double a, int32_t k) { return x64_scaled_round(a, k); }

double permx_x64_to_double(int64_t hi, uint64_t lo, int32_t e) {
    XAcc a;
    a.acc = (__int128)(((unsigned __int128)(uint64_t)hi << 64) | lo);
    a.E = e;
    a.set = true;
    return x64_acc_to_double(a, 0);
}

int permx_x64_product(const int64_t* R, int32_t n, int64_t* m_out, int32_t* e_out) {
    if (!R || !m_out || !e_out || n < 1 || n > 64) return -1;
    XReal t[4];
    for (int q = 0; q < 4 && q < n; ++q) t[q] = x64_head(R[q], q + 4 >= n);
    for (int i = 4; i < n; ++i) t[i & 3] = x64_mul_row(t[i & 3], R[i]);
    const XReal p = x64_term(t, n);
    *m_out = p.m;
    *e_out = p.e;
    return 0;
}

int permx_x64c_product(const int64_t* Rr, const int64_t* Ri, int32_t n, int64_t* re_out, int64_t* im_out,
                       int32_t* e_out) {
    if (!Rr || !Ri || !re_out || !im_out || !e_out || n < 1 || n > 64) return -1;
    XCplx t[4];
    for (int q = 0; q < 4 && q < n; ++q) t[q] = x64c_head(Rr[q], Ri[q], q + 4 >= n);
    for (int i = 4; i < n; ++i) t[i & 3] = x64c_mul_row(t[i & 3], Rr[i], Ri[i]);
    const XCplx p = x64c_term(t, n);
    *re_out = p.re;
    *im_out = p.im;
    *e_out = p.e;
    return 0;
}

int permx_x64_accumulate(const int64_t* m, const int32_t* e, const int32_t* neg, int32_t count, int32_t scale,
                         double* hi, double* lo) {
    if (!m || !e || !neg || !hi || !lo || count < 0 || count > 4096) return -1;
    XAcc a;
    x64_acc_init(a);
    for (int k = 0; k < count; ++k) x64_acc_add(a, m[k], e[k], neg[k] != 0);
    x64_acc_to_dd(a, scale, *hi, *lo);
    return 0;
}

int permx_x64_accumulate_merged(const int64_t* m, const int32_t* e, const int32_t* neg, int32_t count,
                                int32_t parts, int32_t swap, int32_t scale, double* hi, double* lo) {
    if (!m || !e || !neg || !hi || !lo || count < 0 || count > 4096 || parts < 1 || parts > 32 ||
        (parts & (parts - 1)))
        return -1;
    XAcc a[32];
    const int per = (count + parts - 1) / parts;
    for (int q = 0; q < parts; ++q) {
        x64_acc_init(a[q]);
        for (int k = q * per; k < count && k < (q + 1) * per; ++k) x64_acc_add(a[q], m[k], e[k], neg[k] != 0);
    }
    // every "lane" q merges with q ^ d, as the warp butterfly does
    for (int d = 1; d < parts; d <<= 1) {
        XAcc b[32];
        for (int q = 0; q < parts; ++q) {
            b[q] = swap ? a[q ^ d] : a[q];
            x64_acc_merge(b[q], swap ? a[q] : a[q ^ d]);
        }
        for (int q = 0; q < parts; ++q) a[q] = b[q];
    }
    for (int q = 1; q < parts; ++q)
        if (a[q].set != a[0].set || (a[0].set && (a[q].acc != a[0].acc || a[q].E != a[0].E))) return -2;
    x64_acc_to_dd(a[0], scale, *hi, *lo);
    return 0;
}

int permx_plan_describe(int field, const int32_t* n, int64_t batch, int64_t* groups, int32_t max_groups,
                        int64_t* order, int64_t* totals) {
    clear_error();
    if (field != PERMX_FIELD_C128 && field != PERMX_FIELD_F64 && field != PERMX_FIELD_MODP)
        return fail(PERMX_EINVAL, "unknown field");
    if (batch < 1 || !n || !groups || !order || !totals || max_groups < 1) return fail(PERMX_EINVAL, "bad arguments");
    const int max_n = field == PERMX_FIELD_MODP ? PERMX_MAX_N_MODP : PERMX_MAX_N_FP;
    for (int64_t b = 0; b < batch; ++b)
        if (n[b] < 1 || n[b] > max_n) return fail(PERMX_EINVAL, "n out of range");
    const BatchPlan P = plan_batch(n, batch, (Field)field);
    if ((int64_t)P.groups.size() > max_groups) return fail(PERMX_EINVAL, "more groups than max_groups");
    int64_t k = 0;
    for (size_t gi = 0; gi < P.groups.size(); ++gi) {
        const GroupPlan& g = P.groups[gi];
        int64_t* row = groups + gi * PERMX_PLAN_COLS;
        const int64_t v[PERMX_PLAN_COLS] = {g.n, g.ell, g.log2_chunks, g.ld, g.mat_stride, g.col_off, g.items,
                                            g.partials_per_mat, g.part_off, g.x64 ? 1 : 0, (int64_t)g.mats.size()};
        for (int c = 0; c < PERMX_PLAN_COLS; ++c) row[c] = v[c];
        for (int64_t m : g.mats) order[k++] = m;
    }
    totals[0] = P.col_elems;
    totals[1] = P.total_partials;
    return (int)P.groups.size();
}

int permx_arena_run(int64_t capacity, const int64_t* ops, int32_t nops, int64_t* results) {
    clear_error();
    if (capacity < 0 || nops < 0 || (nops > 0 && (!ops || !results))) return fail(PERMX_EINVAL, "bad arguments");
    Arena a;
    a.reset((size_t)capacity);
    std::vector<int64_t> size_of(nops, -1);   // bytes of each live block, by allocating operation
    for (int32_t k = 0; k < nops; ++k) {
        const int64_t kind = ops[2 * k], v = ops[2 * k + 1];
        if (kind == 0) {
            if (v < 0) return fail(PERMX_EINVAL, "negative size");
            results[3 * k] = a.alloc((size_t)v);
            if (results[3 * k] >= 0) size_of[k] = v;
        } else if (kind == 1) {
            if (v < 0 || v >= k || ops[2 * v] != 0 || size_of[v] < 0) return fail(PERMX_EINVAL, "bad release");
            a.release((size_t)results[3 * v], (size_t)size_of[v]);
            size_of[v] = -1;
            results[3 * k] = 0;
        } else {
            return fail(PERMX_EINVAL, "unknown operation");
        }
        results[3 * k + 1] = (int64_t)a.used();
        results[3 * k + 2] = (int64_t)a.largest_free();
    }
    return (int)a.free_blocks();
}

}  // extern "C"
