// Host-side field set-up and Chinese remaindering for the Schur permanent
// (paper §2.1): primes p = 1 (mod n) below 2^31, a primitive n-th root of
// unity g mod p, the residue matrix (g^{jk} mod p), and Garner's mixed-radix
// CRT to the symmetric range.  Integers wider than 64 bits use a small
// little-endian base-2^32 magnitude type.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "field.h"

namespace permx {

uint32_t pow_mod(uint32_t b, uint64_t e, uint32_t p) {
    uint64_t r = 1 % p, x = b % p;
    while (e) {
        if (e & 1) r = r * x % p;
        x = x * x % p;
        e >>= 1;
    }
    return (uint32_t)r;
}

// Deterministic Miller–Rabin: bases 2, 3, 5, 7 decide every n < 3,215,031,751.
bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u}) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint32_t d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; ++s; }
    for (uint32_t a : {2u, 3u, 5u, 7u}) {
        uint64_t x = pow_mod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = x * x % n;
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// Newton's iteration x <- x (2 - p x) doubles the correct low bits each step.
uint32_t inv_mod_2_32(uint32_t p) {
    uint32_t x = p;                     // correct to 3 bits for odd p
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return x;
}

int primes_1_mod_n(int n, int count, int skip, uint32_t* out) {
    if (n < 1 || count < 0 || skip < 0) return -1;
    int found = 0;
    // largest k with k*n + 1 < 2^31
    for (int64_t k = ((int64_t)(1u << 31) - 2) / n; k > 0 && found < count + skip; --k) {
        const uint64_t p = (uint64_t)k * n + 1;
        if (p >= (1ull << 31) || p < 3) continue;
        if (is_prime_u32((uint32_t)p)) {
            if (found >= skip) out[found - skip] = (uint32_t)p;
            ++found;
        }
    }
    return found - skip;
}

static std::vector<uint32_t> prime_factors(uint32_t m) {
    std::vector<uint32_t> f;
    for (uint32_t d = 2; (uint64_t)d * d <= m; ++d) {
        if (m % d == 0) {
            f.push_back(d);
            while (m % d == 0) m /= d;
        }
    }
    if (m > 1) f.push_back(m);
    return f;
}

int primitive_root(uint32_t p, int n, uint32_t* g_out) {
    if (n < 1 || p < 3 || (p - 1) % (uint32_t)n != 0) return -1;
    const std::vector<uint32_t> qs = prime_factors((uint32_t)n);
    for (uint32_t h = 2; h < p; ++h) {
        const uint32_t g = pow_mod(h, (p - 1) / (uint32_t)n, p);
        if (pow_mod(g, (uint64_t)n, p) != 1) continue;
        bool ok = true;
        for (uint32_t q : qs)
            if (pow_mod(g, (uint64_t)(n / q), p) == 1) { ok = false; break; }
        if (ok) { *g_out = g; return 0; }
    }
    return -1;
}

void schur_residues(int n, uint32_t p, uint32_t g, uint32_t* out) {
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) out[j * n + k] = pow_mod(g, (uint64_t)((j * k) % n), p);
}

// ---------------------------------------------------------------------------
// magnitudes in base 2^32
// ---------------------------------------------------------------------------
void Big::trim() {
    while (!w.empty() && w.back() == 0) w.pop_back();
}
void Big::mul_add(uint32_t m, uint32_t a) {
    uint64_t carry = a;
    for (auto& x : w) {
        uint64_t t = (uint64_t)x * m + carry;
        x = (uint32_t)t;
        carry = t >> 32;
    }
    if (carry) w.push_back((uint32_t)carry);
    trim();
}
uint32_t Big::mod(uint32_t p) const {
    uint64_t r = 0;
    for (size_t i = w.size(); i-- > 0;) r = ((r << 32) | w[i]) % p;
    return (uint32_t)r;
}
int Big::cmp(const Big& o) const {
    if (w.size() != o.w.size()) return w.size() < o.w.size() ? -1 : 1;
    for (size_t i = w.size(); i-- > 0;)
        if (w[i] != o.w[i]) return w[i] < o.w[i] ? -1 : 1;
    return 0;
}
Big Big::sub(const Big& o) const {   // requires *this >= o
    Big r = *this;
    int64_t borrow = 0;
    for (size_t i = 0; i < r.w.size(); ++i) {
        int64_t t = (int64_t)r.w[i] - (i < o.w.size() ? o.w[i] : 0) - borrow;
        borrow = t < 0;
        r.w[i] = (uint32_t)(t + (borrow ? (1ll << 32) : 0));
    }
    r.trim();
    return r;
}
Big Big::mul(const Big& o) const {
    Big r;
    r.w.assign(w.size() + o.w.size() + 1, 0);
    for (size_t i = 0; i < w.size(); ++i) {
        uint64_t carry = 0;
        for (size_t j = 0; j < o.w.size(); ++j) {
            uint64_t t = (uint64_t)w[i] * o.w[j] + r.w[i + j] + carry;
            r.w[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        size_t k = i + o.w.size();
        while (carry) {
            uint64_t t = (uint64_t)r.w[k] + carry;
            r.w[k++] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    r.trim();
    return r;
}
std::string Big::decimal() const {
    if (w.empty()) return "0";
    Big t = *this;
    std::vector<uint32_t> parts;   // base 1e9, little-endian
    while (!t.w.empty()) {
        uint64_t r = 0;
        for (size_t i = t.w.size(); i-- > 0;) {
            uint64_t cur = (r << 32) | t.w[i];
            t.w[i] = (uint32_t)(cur / 1000000000u);
            r = cur % 1000000000u;
        }
        t.trim();
        parts.push_back((uint32_t)r);
    }
    std::string s = std::to_string(parts.back());
    char buf[16];
    for (size_t i = parts.size() - 1; i-- > 0;) {
        std::snprintf(buf, sizeof buf, "%09u", parts[i]);
        s += buf;
    }
    return s;
}

// Garner: x = v_0 + v_1 p_0 + v_2 p_0 p_1 + ..., 0 <= v_k < p_k, then the
// symmetric representative in (-M/2, M/2].
void crt_garner(const uint32_t* r, const uint32_t* p, int k, Big& mag, bool& negative) {
    std::vector<uint32_t> v(k);
    for (int i = 0; i < k; ++i) {
        // value of the already-known prefix mod p_i, and prod_{j<i} p_j mod p_i
        uint64_t acc = 0, prod = 1;
        for (int j = 0; j < i; ++j) {
            acc = (acc + (uint64_t)v[j] * prod) % p[i];
            prod = prod * (p[j] % p[i]) % p[i];
        }
        const uint64_t diff = ((uint64_t)r[i] % p[i] + p[i] - acc) % p[i];
        const uint64_t inv = pow_mod((uint32_t)prod, p[i] - 2, p[i]);   // p_i prime
        v[i] = (uint32_t)(diff * inv % p[i]);
    }
    Big x;                                   // Horner from the top digit
    for (int i = k - 1; i >= 0; --i) x.mul_add(p[i], v[i]);
    Big M;
    M.w = {1};
    for (int i = 0; i < k; ++i) M.mul_add(p[i], 0);
    // x > M/2  <=>  2x > M
    Big two_x = x;
    two_x.mul_add(2, 0);
    if (two_x.cmp(M) > 0) {
        mag = M.sub(x);
        negative = true;
    } else {
        mag = x;
        negative = false;
    }
    if (mag.w.empty()) negative = false;
}

// M = prod p > 2 n^{n/2}  <=>  M^2 > 4 n^n, exactly.
bool modulus_suffices(int n, const uint32_t* p, int k) {
    Big M;
    M.w = {1};
    for (int i = 0; i < k; ++i) M.mul_add(p[i], 0);
    Big lhs = M.mul(M);
    Big rhs;
    rhs.w = {4};
    for (int i = 0; i < n; ++i) rhs.mul_add((uint32_t)n, 0);
    return lhs.cmp(rhs) > 0;
}

int schur_prime_count(int n) {
    const double b = (n / 2.0) * std::log2((double)n) + 2.0;
    int k = (int)std::ceil(b / 30.0) + 1;
    std::vector<uint32_t> ps(PERMX_MAX_PRIMES);
    while (k < PERMX_MAX_PRIMES) {
        int got = primes_1_mod_n(n, k, 0, ps.data());
        if (got == k && modulus_suffices(n, ps.data(), k)) break;
        ++k;
    }
    return k;
}

}  // namespace permx
