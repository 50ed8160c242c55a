// Batch planning structures shared by batch.cu, schur.cpp and serve.cpp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace permx {

enum class Field { C128 = 0, F64 = 1, MODP = 2 };

struct StageDesc {          // one matrix to stage column-major (offsets in entries)
    int64_t src;            // A + src: row-major n*n
    int64_t dst;            // colT + dst: column j at + j*ld
    int32_t n, ld;
    uint32_t p;             // F_p only: the prime (x column arithmetic)
    int32_t nw;             // 1: also write x_i = a_{i,n-1} - (1/2) sum_j a_ij as column n
};


struct ModpFinalAt {
    int64_t acc_index, out_index;
    uint32_t p, rfix;
    int32_t negate, pad_;
};


struct GroupPlan {
    int n = 0, ell = 0, log2_chunks = 0, ld = 0, nw = 1;
    bool x64 = false;                // float fields: integer-mantissa walk
    int64_t mat_stride = 0;          // elements (uint32 or double) between matrices
    int64_t col_off = 0;             // elements
    int64_t first_mat = 0;           // index of the group's first matrix in plan order
    int64_t items = 0;               // chunks in the group
    int64_t partials_per_mat = 0;    // fp: partial slots per matrix
    int64_t part_off = 0;            // fp: first partial slot of the group
    std::vector<int64_t> mats;       // batch indices in plan order
};

struct BatchPlan {
    Field field = Field::MODP;
    int64_t batch = 0;
    int64_t col_elems = 0;
    int64_t total_partials = 0;
    std::vector<GroupPlan> groups;
};

// Streams on which the size groups of one batch run concurrently, so that
// the tail of one group's Gray walk overlaps the next group's walk.  A set
// belongs to one host thread (thread_streams) or to one plan, so two threads
// never share a stream and a stream in a graph capture is never used by
// another thread.  fork/join are reused by every execution of the set's owner.
constexpr int kGroupStreams = 8;
struct StreamSet {
    int device = -1;
    cudaStream_t side[kGroupStreams] = {};
    cudaEvent_t fork = nullptr, join[kGroupStreams] = {};
    cudaError_t create(int dev);   // on device dev (which must be current)
    void destroy();
};
// This thread's stream set for the current device (created on first use), or
// nullptr if it could not be created (the groups then run on the call's stream).
StreamSet* thread_streams();

struct Prepared {                   // a planned batch with its workspace (device) and metadata uploaded
    Field field = Field::MODP;
    int64_t batch = 0;
    BatchPlan P;
    bool x64 = false;
    unsigned char* ws = nullptr;
    size_t bytes = 0;
    size_t o_stage = 0, o_p = 0, o_pinv = 0, o_fin = 0, o_meta_end = 0, o_acc = 0, o_col = 0, o_part = 0;
    size_t o_done = 0, o_zero_end = 0;  // [o_done, o_zero_end): finalisation tickets (+ F_p accumulators), zeroed per execution
    std::vector<unsigned char> meta;    // metadata passed by value to the set-up kernel (empty: uploaded once)
    StreamSet* streams = nullptr;       // group streams (nullptr: this thread's set)
};
int prepare_batch(Field field, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                  cudaStream_t s, Prepared& X);
int execute_batch(const Prepared& X, const void* A, void* out, cudaStream_t s);
void release_batch(Prepared& X, cudaStream_t s);
int chunk_log2(Field field, int n, int bits);
int tune_get(int field, int n);
void tune_set(int field, int n, int ell);

int validate_batch(const void* A, const int32_t* n, const int64_t* offset, int64_t batch, const void* out,
                   int max_n);
BatchPlan plan_batch(const int32_t* n, int64_t batch, Field field);
uint64_t plan_units(const BatchPlan& P);
int run_modp_batch(const uint32_t* A, const int32_t* n, const int64_t* offset, const uint32_t* p, int64_t batch,
                   uint32_t* out, cudaStream_t s);
cudaError_t launch_stage(int field, const void* A, const StageDesc* d, int64_t count, void* colT, cudaStream_t s);
cudaError_t launch_stage_x64(bool cplx, const void* A, const StageDesc* d, int64_t count, void* colT,
                             cudaStream_t s);
int set_fp_arith(int mode);
cudaError_t launch_finalize_fp(const double* partial, const FpFinal* f, int64_t count, bool cplx, bool x64, void* out,
                               cudaStream_t s);
cudaError_t launch_finalize_modp_at(const unsigned long long* acc, const ModpFinalAt* f, int64_t count, uint32_t* out,
                                    cudaStream_t s);
int run_fp_batch(const double* A, const int32_t* n, const int64_t* offset, int64_t batch, void* out, bool cplx,
                 cudaStream_t s);

}  // namespace permx
