/*
 * Plain CPU Gray-code Ryser walks — BENCHMARK / TEST INFRASTRUCTURE
 * ONLY (the same rule as oracle.c: only tests/ and the cpu_baseline leg of
 * bench.py load this library; the CUDA product never links, loads or calls
 * it, and it shares no header, helper or constant with the product).
 *
 * What it is: the paper's own CPU algorithm (§2.2, Gray-code blocks) as a
 * plain one-core program, the comparator for the paper's GPU-over-single-
 * threaded-CPU speed-ups.  Unlike oracle.c, which recomputes every row sum
 * for every subset (O(n^2) per subset, obviously correct), these walks keep
 * the row sums r_i and update them with one column per step (O(n) per
 * subset):
 *   subsets g(k) = k XOR (k >> 1) for k in a range [k0, k1); g(k) and g(k-1)
 *   differ in column j = ctz(k); r_i += a_ij when j enters g(k), r_i -= a_ij
 *   when it leaves; the term prod_i r_i enters with sign (-1)^{|g(k)|}.
 * Over [0, 2^n) the signed sum is (-1)^n perm(A) (paper §1, Ryser's formula).
 *
 * Arithmetic is the plainest of each kind: uint64 with '%' for F_p (paper
 * §2.1), IEEE double (or complex double) with no compensation for R and C.
 * No SIMD intrinsics, no blocking: the compiler's -O2 only.  The walks run on
 * one thread; cpuwalk_modp_gray_range_mt splits a range into one contiguous
 * Gray block per OpenMP thread (paper §2.2, as the paper's multi-core CPU
 * comparison does), each walked by the one-thread code.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

static int ctz64(uint64_t x) { return __builtin_ctzll(x); }

/* sum_{k0 <= k < k1} (-1)^{|g(k)|} prod_i sum_{j in g(k)} a_ij  (mod p),
 * A row-major n x n with entries < p, 1 <= n <= 63, k1 <= 2^n. */
int cpuwalk_modp_gray_range(int n, const uint32_t* A, uint32_t p, uint64_t k0, uint64_t k1, uint32_t* out) {
    if (n < 1 || n > 63 || !A || !out || p < 2 || k0 > k1 || k1 > (1ull << n)) return -1;
    const uint64_t pp = p;
    uint64_t r[64];
    uint64_t S = k0 ^ (k0 >> 1);
    for (int i = 0; i < n; ++i) {
        r[i] = 0;
        for (int j = 0; j < n; ++j)
            if (S & (1ull << j)) r[i] = (r[i] + A[i * n + j]) % pp;
    }
    int odd = __builtin_popcountll(S) & 1;
    uint64_t pos = 0, neg = 0;
    for (uint64_t k = k0; k < k1; ++k) {
        if (k > k0) {
            const int j = ctz64(k);
            S ^= 1ull << j;
            odd ^= 1;
            if (S & (1ull << j)) {
                for (int i = 0; i < n; ++i) r[i] = (r[i] + A[i * n + j]) % pp;
            } else {
                for (int i = 0; i < n; ++i) r[i] = (r[i] + pp - A[i * n + j]) % pp;
            }
        }
        uint64_t prod = 1 % pp;
        for (int i = 0; i < n; ++i) prod = prod * r[i] % pp;
        if (odd) neg = (neg + prod) % pp;
        else pos = (pos + prod) % pp;
    }
    *out = (uint32_t)((pos + pp - neg) % pp);
    return 0;
}

/* The same sum with the range cut into nb = omp_get_max_threads() contiguous
 * blocks, shared out by an OpenMP loop (so every block is walked however many
 * threads the runtime grants); the block sums are added mod p in block order.
 * Returns the number of threads that ran (>= 1) or -1. */
int cpuwalk_modp_gray_range_mt(int n, const uint32_t* A, uint32_t p, uint64_t k0, uint64_t k1, uint32_t* out) {
    if (n < 1 || n > 63 || !A || !out || p < 2 || k0 > k1 || k1 > (1ull << n)) return -1;
    const int nb = omp_get_max_threads();
    uint32_t* part = (uint32_t*)calloc((size_t)nb, sizeof(uint32_t));
    if (!part) return -1;
    const uint64_t len = k1 - k0;
    const uint64_t q = len / (uint64_t)nb, r = len % (uint64_t)nb;   // the first r blocks get one more
    int rc = 0, used = 1;
    #pragma omp parallel reduction(|:rc)
    {
        #pragma omp single
        used = omp_get_num_threads();
        #pragma omp for schedule(static, 1)
        for (int t = 0; t < nb; ++t) {
            const uint64_t a = k0 + q * (uint64_t)t + ((uint64_t)t < r ? (uint64_t)t : r);
            const uint64_t b = a + q + ((uint64_t)t < r ? 1 : 0);
            rc |= cpuwalk_modp_gray_range(n, A, p, a, b, &part[t]) != 0;
        }
    }
    uint64_t s = 0;
    for (int t = 0; t < nb; ++t) s = (s + part[t]) % p;
    free(part);
    if (rc) return -1;
    *out = (uint32_t)s;
    return used;
}

/* The same signed sum over real entries in plain double (no (-1)^n factor). */
int cpuwalk_f64_gray_range(int n, const double* A, uint64_t k0, uint64_t k1, double* out) {
    if (n < 1 || n > 63 || !A || !out || k0 > k1 || k1 > (1ull << n)) return -1;
    double r[64];
    uint64_t S = k0 ^ (k0 >> 1);
    for (int i = 0; i < n; ++i) {
        r[i] = 0.0;
        for (int j = 0; j < n; ++j)
            if (S & (1ull << j)) r[i] += A[i * n + j];
    }
    int odd = __builtin_popcountll(S) & 1;
    double acc = 0.0;
    for (uint64_t k = k0; k < k1; ++k) {
        if (k > k0) {
            const int j = ctz64(k);
            S ^= 1ull << j;
            odd ^= 1;
            if (S & (1ull << j)) {
                for (int i = 0; i < n; ++i) r[i] += A[i * n + j];
            } else {
                for (int i = 0; i < n; ++i) r[i] -= A[i * n + j];
            }
        }
        double prod = 1.0;
        for (int i = 0; i < n; ++i) prod *= r[i];
        acc += odd ? -prod : prod;
    }
    *out = acc;
    return 0;
}

/* Complex entries (re, im interleaved, row-major); out = (re, im). */
int cpuwalk_c128_gray_range(int n, const double* A, uint64_t k0, uint64_t k1, double* out) {
    if (n < 1 || n > 63 || !A || !out || k0 > k1 || k1 > (1ull << n)) return -1;
    double rr[64], ri[64];
    uint64_t S = k0 ^ (k0 >> 1);
    for (int i = 0; i < n; ++i) {
        rr[i] = 0.0;
        ri[i] = 0.0;
        for (int j = 0; j < n; ++j) {
            if (!(S & (1ull << j))) continue;
            rr[i] += A[2 * (i * n + j)];
            ri[i] += A[2 * (i * n + j) + 1];
        }
    }
    int odd = __builtin_popcountll(S) & 1;
    double ar = 0.0, ai = 0.0;
    for (uint64_t k = k0; k < k1; ++k) {
        if (k > k0) {
            const int j = ctz64(k);
            S ^= 1ull << j;
            odd ^= 1;
            if (S & (1ull << j)) {
                for (int i = 0; i < n; ++i) {
                    rr[i] += A[2 * (i * n + j)];
                    ri[i] += A[2 * (i * n + j) + 1];
                }
            } else {
                for (int i = 0; i < n; ++i) {
                    rr[i] -= A[2 * (i * n + j)];
                    ri[i] -= A[2 * (i * n + j) + 1];
                }
            }
        }
        double pr = 1.0, pi = 0.0;
        for (int i = 0; i < n; ++i) {
            const double t = pr * rr[i] - pi * ri[i];
            pi = pr * ri[i] + pi * rr[i];
            pr = t;
        }
        if (odd) {
            ar -= pr;
            ai -= pi;
        } else {
            ar += pr;
            ai += pi;
        }
    }
    out[0] = ar;
    out[1] = ai;
    return 0;
}
