// Schur-permanent run structures (schur.cpp) and the single-matrix F_p
// range runner shared with the serving loop.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "field.h"

namespace permx {

cudaError_t stage_columns_u32(const uint32_t* A, int n, int ld, uint32_t p, int nw, uint32_t* colT,
                              cudaStream_t s);

// One staged F_p matrix, summed over windows of Gray indices.  nw = 0: plain
// Ryser over 2^n subsets; nw = 1: Nijenhuis-Wilf form over 2^(n-1) subsets.
struct ModpRange {
    int n = 0, ell = 0, ld = 0, nw = 0, bits = 0;
    uint32_t p = 0;
    cudaStream_t s = nullptr;
    uint32_t* col = nullptr;          // column-major copy + accumulator
    uint32_t* params = nullptr;       // {p, p^-1 mod 2^32}
    unsigned long long* acc = nullptr;
    // window > 0: the walks will cover windows of about `window` Gray indices;
    // the chunk is shortened (to no less than 2^8 steps) so that a window
    // still holds 2^19 chunks, several per resident thread.
    int init(const uint32_t* A_dev, int n, uint32_t p, int nw, cudaStream_t s, uint64_t window = 0);
    int run(uint64_t k0, uint64_t k1, uint32_t* residue);   // synchronous
    void release();
};

struct SchurState {
    int n = 0;
    std::vector<uint32_t> primes;     // main primes then the check prime
    std::vector<uint32_t> done;       // residues of perm(S_n) for the finished primes, in order
    uint64_t cursor = 0;              // next Gray index of the current prime
    uint32_t partial = 0;             // signed sum over Gray indices [0, cursor) mod p (Nijenhuis-Wilf form,
                                      // without its factor 2 (-1)^(n-1))
};

struct SchurResult {
    std::vector<uint32_t> primes, residues;
    Big magnitude;
    bool negative = false;
};

int write_checkpoint(const std::string& path, const SchurState& st);
int read_checkpoint(const std::string& path, SchurState& st);
int schur_crt_run(int n, int nprimes, const char* ckpt_path, uint64_t slice_subsets, int64_t max_slices,
                  SchurResult& res);
// the same with the caller's primes (the last one is the check prime)
int schur_crt_run_primes(int n, const std::vector<uint32_t>& primes, const char* ckpt_path, uint64_t slice_subsets,
                         int64_t max_slices, SchurResult& res);

// one shard of a strong split over GPUs (see perm_schur_shard)
int schur_shard(int n, const std::vector<uint32_t>& primes, int slices, int shard, int nshards,
                std::vector<uint32_t>& partial);

}  // namespace permx
