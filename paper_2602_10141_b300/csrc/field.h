// Host field helpers for the Schur permanent (paper §2.1).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace permx {

struct Big {                         // non-negative integer, base 2^32, little-endian
    std::vector<uint32_t> w;
    void trim();
    void mul_add(uint32_t m, uint32_t a);   // *this = *this * m + a
    uint32_t mod(uint32_t p) const;
    int cmp(const Big& o) const;
    Big sub(const Big& o) const;
    Big mul(const Big& o) const;
    std::string decimal() const;
};

int primes_1_mod_n(int n, int count, int skip, uint32_t* out);
int primitive_root(uint32_t p, int n, uint32_t* g_out);
void schur_residues(int n, uint32_t p, uint32_t g, uint32_t* out);
void crt_garner(const uint32_t* r, const uint32_t* p, int k, Big& mag, bool& negative);
bool modulus_suffices(int n, const uint32_t* p, int k);
int schur_prime_count(int n);

}  // namespace permx
