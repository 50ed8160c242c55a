/*
 * Plain CPU oracle for matrix permanents — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg
 * of bench.py may load this library.  The product path (the CUDA library
 * under paper_2602_10141_b300/) never links, loads or calls it, and this
 * file shares no header, helper, table or constant with it.
 *
 * Everything here is deliberately slow and direct:
 *
 *  - perm by the definition  perm(A) = sum_{sigma in S_n} prod_i a_{i,sigma(i)}
 *    (paper §1, the displayed definition), either by brute force over all n!
 *    permutations (small n) or by the same sum organised as an expansion
 *    along rows memoised over the set of columns already used ("row
 *    expansion DP": f(T) = sum over bijections rows {0..|T|-1} -> T of the
 *    product of the chosen entries; f({all}) = perm(A)).
 *  - perm by Ryser's inclusion-exclusion formula, in the sign convention
 *       perm(A) = (-1)^n sum_{S subset [n]} (-1)^{|S|} prod_i sum_{j in S} a_ij
 *    (the formula the paper cites in §1 and evaluates in §2.1-2.2), by
 *    direct enumeration of the subsets S with every row sum recomputed from
 *    scratch: no Gray code, no incremental update.
 *  - F_p versions of both with uint64 arithmetic and the C '%' operator
 *    (paper §2.1: the permanent of (g^{jk} mod p) over Z/pZ).
 *  - Counts c_m = #{sigma : sum_i i*sigma(i) = m (mod n)}: the definition
 *    applied to the Schur matrix S_n = (w^{jk}) in Z[x]/(x^n - 1) with w -> x,
 *    so that perm(S_n) = sum_m c_m w^m (paper §1, Schur matrix; §2.1).
 *
 * Real and complex values are carried in double-double ("dd") arithmetic
 * built from Knuth's TwoSum and the FMA-based TwoProduct (error-free
 * transformations from the published literature), about 106 significant
 * bits, so that the oracle's own rounding is far below any tolerance the
 * tests apply to the GPU path.  Brute force uses long double.
 *
 * Compile with -O2 -fopenmp -ffp-contract=off and never with -ffast-math:
 * the error-free transformations depend on exact IEEE rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

/* ------------------------------------------------------------------ */
/* double-double arithmetic                                             */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } cdd;

/* Knuth's TwoSum: s + e == a + b exactly. */
static inline dd two_sum(double a, double b) {
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    dd r = { s, (a - av) + (b - bv) };
    return r;
}
/* Dekker's Fast2Sum, valid when |a| >= |b| (or a == 0). */
static inline dd fast_two_sum(double a, double b) {
    double s = a + b;
    dd r = { s, b - (s - a) };
    return r;
}
/* TwoProduct with a fused multiply-add: p + e == a * b exactly. */
static inline dd two_prod(double a, double b) {
    double p = a * b;
    dd r = { p, fma(a, b, -p) };
    return r;
}
static inline dd dd_from(double a) { dd r = { a, 0.0 }; return r; }
static inline dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static inline dd dd_neg(dd a) { dd r = { -a.hi, -a.lo }; return r; }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static inline dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
static inline cdd cdd_add(cdd a, cdd b) { cdd r = { dd_add(a.re, b.re), dd_add(a.im, b.im) }; return r; }
static inline cdd cdd_sub(cdd a, cdd b) { cdd r = { dd_sub(a.re, b.re), dd_sub(a.im, b.im) }; return r; }
static inline cdd cdd_mul(cdd a, cdd b) {
    cdd r = { dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)),
              dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re)) };
    return r;
}
static inline cdd cdd_zero(void) { cdd r = { {0.0, 0.0}, {0.0, 0.0} }; return r; }
static inline double dd_to_d(dd a) { return a.hi + a.lo; }

static inline int popcount64(uint64_t x) { return __builtin_popcountll(x); }

#define ORACLE_MAX_N_FP 30
#define ORACLE_MAX_N_MODP 48

/* ------------------------------------------------------------------ */
/* Brute force over all n! permutations (definition, paper §1).         */
/* Recursion assigns row `row` to every unused column in turn.           */
/* ------------------------------------------------------------------ */
static long double brute_r_rec(int n, const double* A, int row, uint32_t used, long double prod) {
    if (row == n) return prod;
    long double s = 0.0L;
    for (int j = 0; j < n; ++j) {
        if (used & (1u << j)) continue;
        s += brute_r_rec(n, A, row + 1, used | (1u << j), prod * (long double)A[row * n + j]);
    }
    return s;
}

/* perm of a real row-major n x n matrix, n <= 11; out[0] + out[1] = value. */
int oracle_perm_brute_r(int n, const double* A, double* out) {
    if (n < 1 || n > 11 || !A || !out) return -1;
    long double v = brute_r_rec(n, A, 0, 0u, 1.0L);
    out[0] = (double)v;
    out[1] = (double)(v - (long double)out[0]);
    return 0;
}

static void brute_c_rec(int n, const double* A, int row, uint32_t used,
                        long double pr, long double pi, long double* sr, long double* si) {
    if (row == n) { *sr += pr; *si += pi; return; }
    for (int j = 0; j < n; ++j) {
        if (used & (1u << j)) continue;
        long double ar = A[2 * (row * n + j)], ai = A[2 * (row * n + j) + 1];
        brute_c_rec(n, A, row + 1, used | (1u << j), pr * ar - pi * ai, pr * ai + pi * ar, sr, si);
    }
}

/* perm of a complex row-major matrix (interleaved re, im), n <= 11;
 * out = {re_hi, re_lo, im_hi, im_lo}. */
int oracle_perm_brute_c(int n, const double* A, double* out) {
    if (n < 1 || n > 11 || !A || !out) return -1;
    long double sr = 0.0L, si = 0.0L;
    brute_c_rec(n, A, 0, 0u, 1.0L, 0.0L, &sr, &si);
    out[0] = (double)sr; out[1] = (double)(sr - (long double)out[0]);
    out[2] = (double)si; out[3] = (double)(si - (long double)out[2]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Row-expansion DP (definition, paper §1): f[T] for column sets T.      */
/* f[empty] = 1;  f[T] = sum_{j in T} f[T \ {j}] * a_{|T|-1, j}.         */
/* Layers |T| = 1..n are processed in order; within a layer the masks   */
/* are independent and are split across OpenMP threads.                 */
/* ------------------------------------------------------------------ */
int oracle_perm_dp_r(int n, const double* A, double* out) {
    if (n < 1 || n > 26 || !A || !out) return -1;
    uint64_t full = (1ull << n);
    dd* f = (dd*)malloc(sizeof(dd) * full);
    if (!f) return -2;
    f[0] = dd_from(1.0);
    for (int k = 1; k <= n; ++k) {
        const double* arow = A + (size_t)(k - 1) * n;
        #pragma omp parallel for schedule(static)
        for (int64_t T = 1; T < (int64_t)full; ++T) {
            if (popcount64((uint64_t)T) != k) continue;
            dd s = dd_from(0.0);
            for (int j = 0; j < n; ++j)
                if ((uint64_t)T & (1ull << j))
                    s = dd_add(s, dd_mul(f[(uint64_t)T & ~(1ull << j)], dd_from(arow[j])));
            f[T] = s;
        }
    }
    out[0] = f[full - 1].hi;
    out[1] = f[full - 1].lo;
    free(f);
    return 0;
}

int oracle_perm_dp_c(int n, const double* A, double* out) {
    if (n < 1 || n > 25 || !A || !out) return -1;
    uint64_t full = (1ull << n);
    cdd* f = (cdd*)malloc(sizeof(cdd) * full);
    if (!f) return -2;
    f[0] = cdd_zero();
    f[0].re = dd_from(1.0);
    for (int k = 1; k <= n; ++k) {
        const double* arow = A + 2 * (size_t)(k - 1) * n;
        #pragma omp parallel for schedule(static)
        for (int64_t T = 1; T < (int64_t)full; ++T) {
            if (popcount64((uint64_t)T) != k) continue;
            cdd s = cdd_zero();
            for (int j = 0; j < n; ++j) {
                if (!((uint64_t)T & (1ull << j))) continue;
                cdd a = { dd_from(arow[2 * j]), dd_from(arow[2 * j + 1]) };
                s = cdd_add(s, cdd_mul(f[(uint64_t)T & ~(1ull << j)], a));
            }
            f[T] = s;
        }
    }
    out[0] = f[full - 1].re.hi; out[1] = f[full - 1].re.lo;
    out[2] = f[full - 1].im.hi; out[3] = f[full - 1].im.lo;
    free(f);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ryser's formula by direct enumeration of S = 1 .. 2^n - 1 in binary   */
/* order, row sums recomputed from scratch for every S.                 */
/* Per-thread partial sums are combined in thread order (deterministic). */
/* abs_terms (optional) receives sum_S |prod_i r_i(S)| in double, the    */
/* magnitude of the terms that cancel, used to scale FP tolerances.     */
/* ------------------------------------------------------------------ */
int oracle_perm_ryser_r(int n, const double* A, double* out, double* abs_terms) {
    if (n < 1 || n > ORACLE_MAX_N_FP || !A || !out) return -1;
    int nt = omp_get_max_threads();
    dd* part = (dd*)calloc((size_t)nt, sizeof(dd));
    double* pabs = (double*)calloc((size_t)nt, sizeof(double));
    if (!part || !pabs) { free(part); free(pabs); return -2; }
    int64_t full = (int64_t)1 << n;
    #pragma omp parallel
    {
        int t = omp_get_thread_num();
        dd acc = dd_from(0.0);
        double aacc = 0.0;
        #pragma omp for schedule(static)
        for (int64_t S = 1; S < full; ++S) {
            dd prod = dd_from(1.0);
            for (int i = 0; i < n; ++i) {
                dd r = dd_from(0.0);
                for (int j = 0; j < n; ++j)
                    if ((uint64_t)S & (1ull << j)) r = dd_add(r, dd_from(A[i * n + j]));
                prod = dd_mul(prod, r);
            }
            aacc += fabs(dd_to_d(prod));
            if (popcount64((uint64_t)S) & 1) acc = dd_sub(acc, prod);
            else acc = dd_add(acc, prod);
        }
        part[t] = acc;
        pabs[t] = aacc;
    }
    dd s = dd_from(0.0);
    double a = 0.0;
    for (int t = 0; t < nt; ++t) { s = dd_add(s, part[t]); a += pabs[t]; }
    if (n & 1) s = dd_neg(s);
    out[0] = s.hi; out[1] = s.lo;
    if (abs_terms) *abs_terms = a;
    free(part); free(pabs);
    return 0;
}

int oracle_perm_ryser_c(int n, const double* A, double* out, double* abs_terms) {
    if (n < 1 || n > ORACLE_MAX_N_FP || !A || !out) return -1;
    int nt = omp_get_max_threads();
    cdd* part = (cdd*)calloc((size_t)nt, sizeof(cdd));
    double* pabs = (double*)calloc((size_t)nt, sizeof(double));
    if (!part || !pabs) { free(part); free(pabs); return -2; }
    int64_t full = (int64_t)1 << n;
    #pragma omp parallel
    {
        int t = omp_get_thread_num();
        cdd acc = cdd_zero();
        double aacc = 0.0;
        #pragma omp for schedule(static)
        for (int64_t S = 1; S < full; ++S) {
            cdd prod = cdd_zero();
            prod.re = dd_from(1.0);
            for (int i = 0; i < n; ++i) {
                cdd r = cdd_zero();
                for (int j = 0; j < n; ++j) {
                    if (!((uint64_t)S & (1ull << j))) continue;
                    r.re = dd_add(r.re, dd_from(A[2 * (i * n + j)]));
                    r.im = dd_add(r.im, dd_from(A[2 * (i * n + j) + 1]));
                }
                prod = cdd_mul(prod, r);
            }
            aacc += hypot(dd_to_d(prod.re), dd_to_d(prod.im));
            if (popcount64((uint64_t)S) & 1) acc = cdd_sub(acc, prod);
            else acc = cdd_add(acc, prod);
        }
        part[t] = acc;
        pabs[t] = aacc;
    }
    cdd s = cdd_zero();
    double a = 0.0;
    for (int t = 0; t < nt; ++t) { s = cdd_add(s, part[t]); a += pabs[t]; }
    if (n & 1) { s.re = dd_neg(s.re); s.im = dd_neg(s.im); }
    out[0] = s.re.hi; out[1] = s.re.lo; out[2] = s.im.hi; out[3] = s.im.lo;
    if (abs_terms) *abs_terms = a;
    free(part); free(pabs);
    return 0;
}

/* ------------------------------------------------------------------ */
/* F_p (paper §2.1).  Entries must be < p; p < 2^32.  uint64 and '%'.     */
/* ------------------------------------------------------------------ */
static uint64_t brute_p_rec(int n, const uint32_t* A, uint64_t p, int row, uint64_t used, uint64_t prod) {
    if (row == n) return prod;
    uint64_t s = 0;
    for (int j = 0; j < n; ++j) {
        if (used & (1ull << j)) continue;
        s = (s + brute_p_rec(n, A, p, row + 1, used | (1ull << j), (prod * A[row * n + j]) % p)) % p;
    }
    return s;
}

int oracle_perm_brute_modp(int n, const uint32_t* A, uint32_t p, uint32_t* out) {
    if (n < 1 || n > 11 || !A || !out || p < 2) return -1;
    *out = (uint32_t)brute_p_rec(n, A, p, 0, 0ull, 1ull % p);
    return 0;
}

int oracle_perm_dp_modp(int n, const uint32_t* A, uint32_t p, uint32_t* out) {
    if (n < 1 || n > 28 || !A || !out || p < 2) return -1;
    uint64_t full = 1ull << n;
    uint32_t* f = (uint32_t*)malloc(sizeof(uint32_t) * full);
    if (!f) return -2;
    f[0] = (uint32_t)(1ull % p);
    for (int k = 1; k <= n; ++k) {
        const uint32_t* arow = A + (size_t)(k - 1) * n;
        #pragma omp parallel for schedule(static)
        for (int64_t T = 1; T < (int64_t)full; ++T) {
            if (popcount64((uint64_t)T) != k) continue;
            uint64_t s = 0;
            for (int j = 0; j < n; ++j)
                if ((uint64_t)T & (1ull << j))
                    s = (s + (uint64_t)f[(uint64_t)T & ~(1ull << j)] * arow[j]) % p;
            f[T] = (uint32_t)s;
        }
    }
    *out = f[full - 1];
    free(f);
    return 0;
}

/* Signed Ryser partial sum over the subsets S = g(k) = k XOR (k >> 1)
 * (the reflected binary Gray code) for k in [k0, k1):
 *     out = sum_k (-1)^{|g(k)|} prod_i sum_{j in g(k)} a_ij   (mod p),
 * with no (-1)^n factor.  Over the full range [0, 2^n) this is
 * (-1)^n perm(A); the Gray map is a bijection of [0, 2^n).  Row sums are
 * recomputed from scratch for every subset. */
int oracle_perm_ryser_modp_gray_range(int n, const uint32_t* A, uint32_t p,
                                      uint64_t k0, uint64_t k1, uint32_t* out) {
    if (n < 1 || n > ORACLE_MAX_N_MODP || !A || !out || p < 2) return -1;
    if (k1 > (1ull << n) || k0 > k1) return -1;
    uint64_t pp = p;
    uint64_t pos = 0, neg = 0;
    #pragma omp parallel for schedule(static) reduction(+:pos, neg)
    for (int64_t kk = (int64_t)k0; kk < (int64_t)k1; ++kk) {
        uint64_t k = (uint64_t)kk;
        uint64_t S = k ^ (k >> 1);
        uint64_t prod = 1 % pp;
        for (int i = 0; i < n; ++i) {
            uint64_t r = 0;
            for (int j = 0; j < n; ++j)
                if (S & (1ull << j)) r = (r + A[i * n + j]) % pp;
            prod = (prod * r) % pp;
        }
        if (popcount64(S) & 1) neg = (neg + prod) % pp; else pos = (pos + prod) % pp;
    }
    *out = (uint32_t)((pos % pp + pp - neg % pp) % pp);
    return 0;
}

/* perm(A) mod p by Ryser's formula over all subsets in binary order. */
int oracle_perm_ryser_modp(int n, const uint32_t* A, uint32_t p, uint32_t* out) {
    if (n < 1 || n > ORACLE_MAX_N_MODP || !A || !out || p < 2) return -1;
    uint64_t pp = p;
    uint64_t pos = 0, neg = 0;
    int64_t full = (int64_t)1 << n;
    #pragma omp parallel for schedule(static) reduction(+:pos, neg)
    for (int64_t SS = 1; SS < full; ++SS) {
        uint64_t S = (uint64_t)SS;
        uint64_t prod = 1 % pp;
        for (int i = 0; i < n; ++i) {
            uint64_t r = 0;
            for (int j = 0; j < n; ++j)
                if (S & (1ull << j)) r = (r + A[i * n + j]) % pp;
            prod = (prod * r) % pp;
        }
        if (popcount64(S) & 1) neg = (neg + prod) % pp; else pos = (pos + prod) % pp;
    }
    uint64_t s = (pos % pp + pp - neg % pp) % pp;
    if (n & 1) s = (pp - s) % pp;
    *out = (uint32_t)s;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Schur-matrix counts: c_m = #{sigma in S_n : sum_i i*sigma(i) = m mod n}. */
/* Row-expansion DP over (column set T, residue r); row k = |T|-1 placed  */
/* in column j contributes k*j.  n <= 20 keeps every count below 2^64    */
/* (sum_m c_m = n! < 2^64 for n <= 20).  out has n entries.              */
/* ------------------------------------------------------------------ */
int oracle_schur_counts(int n, uint64_t* out) {
    if (n < 1 || n > 20 || !out) return -1;
    uint64_t full = 1ull << n;
    uint64_t* f = (uint64_t*)calloc(full * (uint64_t)n, sizeof(uint64_t));
    if (!f) return -2;
    f[0] = 1;   /* T = empty, residue 0 */
    for (int k = 1; k <= n; ++k) {
        int row = k - 1;
        #pragma omp parallel for schedule(static)
        for (int64_t T = 1; T < (int64_t)full; ++T) {
            if (popcount64((uint64_t)T) != k) continue;
            uint64_t* dst = f + (uint64_t)T * n;
            for (int j = 0; j < n; ++j) {
                if (!((uint64_t)T & (1ull << j))) continue;
                const uint64_t* src = f + ((uint64_t)T & ~(1ull << j)) * n;
                int shift = (row * j) % n;
                for (int r = 0; r < n; ++r) dst[(r + shift) % n] += src[r];
            }
        }
    }
    memcpy(out, f + (full - 1) * n, sizeof(uint64_t) * n);
    free(f);
    return 0;
}

int oracle_num_threads(void) { return omp_get_max_threads(); }
/* threads for the following parallel loops (k >= 1) */
void oracle_set_num_threads(int k) { if (k >= 1) omp_set_num_threads(k); }
