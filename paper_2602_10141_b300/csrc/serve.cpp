// Serving: continuous batching of permanent requests (include/permx.h,
// serve_*).  A worker thread runs steps.  Each step
//   1. admits queued requests in arrival order while resident slots, the
//      device-memory arena and the outstanding-work budget allow (a request
//      whose work does not fit lets smaller ones behind it pass, for a
//      bounded time),
//   2. stages the newly admitted matrices column-major in the arena,
//   3. grants every resident request a share of its (field, n) class's wave
//      of Gray-code chunks, in whole lane groups (every request at least one
//      group, then the oldest first), and launches one segment-mode Ryser
//      kernel per class on side streams,
//   4. finalises the requests whose last chunk ran in this step and copies
//      their results back.
// Two steps are in flight: while step k runs on the GPU the worker admits,
// plans and enqueues step k+1 into the other of two buffer sets, and reads
// step k's results once its end event has completed.  Steps stay ordered on
// the server's stream, so a step's staging never overwrites arena space that
// an earlier step still reads.
//
// A request is cut into exactly the chunks and lane groups of the batched
// path and its partial slots are summed by the same fixed-order finalize
// kernel, so its result is bit-identical to perm_c128 / perm_f64 / perm_modp
// on that matrix, alone or in any mix.
//
// plain_fifo = 1 is the baseline: one request at a time, each as its own
// batched call of one matrix, synchronously.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "batch.h"
#include "common.cuh"
#include "permx.h"

namespace permx {
namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Request {
    uint64_t ticket = 0;
    int field = 0, n = 0;
    uint32_t p = 0;
    std::vector<unsigned char> host;   // row-major matrix
    int ell = 0, log2_chunks = 0, lg = 0, ld = 0;
    bool x64 = false;                  // float fields: integer-mantissa walk
    uint64_t chunks = 0, next_chunk = 0;
    double cost = 0.0;                 // work of the whole walk (complex128-term equivalents)
    int64_t arena_off = -1;            // columns, then partial slots / accumulator
    size_t bytes = 0, col_bytes = 0;
    bool finalizing = false;           // its finalize has been enqueued
    bool done = false;
    unsigned char result[16] = {0};
    int64_t t_submit = 0, t_done = 0;
};

int entry_bytes(int field) { return field == PERMX_FIELD_C128 ? 16 : field == PERMX_FIELD_F64 ? 8 : 4; }

// Relative GPU cost of one Gray-walk term (one subset x one row) per field,
// complex128 = 1, from the measured term rates of the walk kernels on B300:
// integer-mantissa walks 2.65e11 (complex) and 8.2e11 (real) terms/s, FP64
// walks 7.8e10 and 1.85e11, the F_p walk 2.7e12.
double term_cost(int field, bool x64) {
    if (field == PERMX_FIELD_MODP) return 0.1;
    if (field == PERMX_FIELD_C128) return x64 ? 1.0 : 3.4;
    return x64 ? 0.32 : 1.4;
}

// A step's buffers: pinned host and device copies of its metadata (staging
// descriptors, segment tables, finalize descriptors, then the results the
// finalize kernels write and the step copies back), the uploaded matrices,
// and the events that bracket the step on the server's stream.
struct StepBuf {
    unsigned char *h_meta = nullptr, *d_meta = nullptr;
    size_t h_meta_cap = 0, d_meta_cap = 0;
    unsigned char *h_upload = nullptr, *d_upload = nullptr;
    size_t h_upload_cap = 0, d_upload_cap = 0;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    bool busy = false;
    double work = 0.0;                                   // work of the chunks this step runs
    std::vector<std::pair<Request*, size_t>> results;   // finished request, offset of its result in h_meta
};

}  // namespace
}  // namespace permx

using namespace permx;

constexpr int kSideStreams = 4;
constexpr int64_t kDefaultWorkBudget = (int64_t)1 << 35;
constexpr int64_t kBypassNs = 20'000'000;   // how long a request that does not fit lets others pass
constexpr size_t kAdmitLookahead = 1024;     // queued requests examined per admission

struct perm_server {
    perm_serve_cfg cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t side[kSideStreams] = {nullptr};
    cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_side[2][kSideStreams] = {};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<Request*> pending;
    std::vector<Request*> resident;
    std::unordered_map<uint64_t, Request*> live;   // every ticket not yet reported done by a poll
    int64_t submitted = 0, completed = 0;
    double resident_work = 0.0;        // work admitted and not yet run by a completed step
    std::atomic<int64_t> steps{0}, launches{0};
    double gpu_busy_ms = 0.0;
    int64_t t_create = 0;
    int worker_error = 0;
    bool x64 = true;                   // float arithmetic fixed when the server is created
    std::string worker_msg;
    // device buffers and state owned by the worker
    unsigned char* arena_base = nullptr;
    Arena arena;
    StepBuf buf[2];
    unsigned char* d_plain = nullptr;  // plain FIFO: the request's matrix and result
    size_t d_plain_cap = 0;
};

namespace {

int grow_device(unsigned char** p, size_t* cap, size_t need) {
    if (need <= *cap) return PERMX_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    size_t c = std::max(need, *cap * 2);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), c);
    if (e != cudaSuccess) {
        *cap = 0;
        return cuda_fail(e, "server buffer");
    }
    *cap = c;
    return PERMX_OK;
}

int grow_pinned(unsigned char** p, size_t* cap, size_t need) {
    if (need <= *cap) return PERMX_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    size_t c = std::max(need, *cap * 2);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(p), c);
    if (e != cudaSuccess) {
        *cap = 0;
        return cuda_fail(e, "server pinned buffer");
    }
    *cap = c;
    return PERMX_OK;
}

void plan_request(Request* r, bool x64) {
    const bool modp = r->field == PERMX_FIELD_MODP;
    // the batched path's plan: Nijenhuis-Wilf form, same chunking
    const int bits = walk_bits(r->n, 1);
    r->ell = chunk_log2((Field)r->field, r->n, bits);
    r->log2_chunks = bits - r->ell;
    r->x64 = !modp && x64;
    r->lg = group_log2(r->log2_chunks, chunks_per_warp(r->x64, r->field == PERMX_FIELD_C128, r->n));
    r->chunks = 1ull << r->log2_chunks;
    r->ld = modp ? pad4(r->n) : r->field == PERMX_FIELD_F64 ? pad2(r->n) : r->n;
    // staged columns (plus the x column); the integer-mantissa layout adds a scale word pair
    r->col_bytes = align256((size_t)(r->n + 1) * r->ld * entry_bytes(r->field) + (r->x64 ? 16 : 0));
    const size_t tail = modp ? 8 : (size_t)(r->chunks >> r->lg) * 8 * fp_slot_doubles(r->x64, r->field == PERMX_FIELD_C128);
    r->bytes = r->col_bytes + align256(tail);
    r->cost = (double)r->n * std::ldexp(1.0, bits) * term_cost(r->field, r->x64);
}

// Admission (under the lock).  Queued requests are taken in arrival order
// while the resident count, the arena and the work budget allow.  A request
// whose work does not fit the budget is skipped and smaller ones behind it may
// pass, until it has waited kBypassNs; then admission stops at it until it
// fits, or until nothing else is resident.  Memory: the first request that
// does not fit the arena stops admission (it keeps its place).
void admit(perm_server* S, std::vector<Request*>& admitted) {
    const double budget = S->cfg.work_budget < 0 ? HUGE_VAL : (double)S->cfg.work_budget;
    const int64_t now = now_ns();
    size_t i = 0;
    while (i < S->pending.size() && i < kAdmitLookahead && (int64_t)S->resident.size() < S->cfg.max_resident) {
        Request* r = S->pending[i];
        const bool fits = S->resident.empty() || S->resident_work + r->cost <= budget;
        if (!fits) {
            if (now - r->t_submit >= kBypassNs) break;   // it has waited long enough: nothing passes it
            ++i;
            continue;
        }
        const int64_t off = S->arena.alloc(r->bytes);
        if (off < 0) break;   // memory-bound admission: wait for residents to finish
        r->arena_off = off;
        S->pending.erase(S->pending.begin() + (std::ptrdiff_t)i);
        S->resident.push_back(r);
        S->resident_work += r->cost;
        admitted.push_back(r);
    }
}

bool has_grantable(const perm_server* S) {
    for (const Request* r : S->resident)
        if (r->next_chunk < r->chunks) return true;
    return false;
}

// Plan and enqueue one step into buffer set B.  Runs on the worker thread;
// the lock is taken only around the shared work counter.
int enqueue_step(perm_server* S, StepBuf& B, int slot, const std::vector<Request*>& admitted) {
    cudaStream_t st = S->stream;
    B.results.clear();
    // ---- grants -------------------------------------------------------------------------
    // A chunk is one thread's Gray walk; a wave is one chunk for every
    // resident thread of the class kernel.  The class kernels of a step share
    // the SMs one after another, so a step lasts about the sum of their wave
    // times, and a class with short chunks would progress one short wave per
    // long step.  Per step every (field, n) class therefore gets as many
    // waves as fit in the longest single-wave time of the step (at most 16),
    // or chunks_per_step chunks in total when set.  Within a class every
    // request first gets a fair share (at least one lane group), then the
    // rest goes to the oldest requests first.
    std::vector<Request*> act;
    for (Request* r : S->resident)
        if (r->next_chunk < r->chunks) act.push_back(r);   // admission order
    std::vector<uint64_t> grant(act.size(), 0);
    std::map<std::pair<int, int>, std::vector<size_t>> by_class;
    for (size_t i = 0; i < act.size(); ++i) by_class[{act[i]->field, act[i]->n}].push_back(i);
    const int64_t fixed = S->cfg.chunks_per_step;
    // one chunk's time on its lane(s), in complex128-term units: 2^ell steps of n terms
    auto chunk_time = [](const Request* r) {
        const int lanes = chunks_per_warp(r->x64, r->field == PERMX_FIELD_C128, r->n) == 16 ? 2 : 1;
        return std::ldexp(1.0, r->ell) * r->n * term_cost(r->field, r->x64) / lanes;
    };
    double longest = 0.0;
    for (auto& kv : by_class) longest = std::max(longest, chunk_time(act[kv.second[0]]));
    for (auto& kv : by_class) {
        const std::vector<size_t>& idx = kv.second;
        Request* r0 = act[idx[0]];
        const int kind = r0->field == PERMX_FIELD_MODP ? 0
                         : r0->field == PERMX_FIELD_F64 ? (r0->x64 ? 3 : 1) : (r0->x64 ? 4 : 2);
        const int64_t waves = std::min<int64_t>(16, std::max<int64_t>(1, (int64_t)(longest / chunk_time(r0))));
        int64_t budget = fixed > 0 ? std::max<int64_t>(1, fixed / (int64_t)by_class.size())
                                   : (int64_t)sm_count() * dispatch_blocks_per_sm(kind, r0->n) * kRyserThreads * waves;
        const int64_t share = budget / (2 * (int64_t)idx.size());
        for (size_t i : idx) {
            const uint64_t G = 1ull << act[i]->lg;
            const uint64_t rem = act[i]->chunks - act[i]->next_chunk;
            grant[i] = std::min(std::max<uint64_t>(G, (uint64_t)share / G * G), rem);
            budget -= (int64_t)grant[i];
        }
        for (size_t i : idx) {
            if (budget <= 0) break;
            const uint64_t G = 1ull << act[i]->lg;
            const uint64_t rem = act[i]->chunks - act[i]->next_chunk - grant[i];
            const uint64_t extra = std::min<uint64_t>(rem, (uint64_t)budget / G * G);
            grant[i] += extra;
            budget -= (int64_t)extra;
        }
    }
    std::map<std::pair<int, int>, std::vector<size_t>> classes;
    for (size_t i = 0; i < act.size(); ++i)
        if (grant[i]) classes[{act[i]->field, act[i]->n}].push_back(i);

    // ---- host metadata: staging descriptors, segment tables, finalize descriptors --------
    std::vector<StageDesc> sd[3], sx[2];   // sx: integer-mantissa staging [complex, real]
    size_t up = 0;
    for (Request* r : admitted) up += align256(r->host.size());
    {
        size_t o = 0;
        for (Request* r : admitted) {
            const int eb = entry_bytes(r->field);
            const StageDesc d{(int64_t)(o / eb), (int64_t)(r->arena_off / eb), r->n, r->ld, r->p, 1};
            if (r->x64) sx[r->field == PERMX_FIELD_C128 ? 0 : 1].push_back(d);
            else sd[r->field].push_back(d);
            o += align256(r->host.size());
        }
    }
    struct L { int field, n; size_t off; int nseg; uint64_t items; Request* any; };
    std::vector<L> launches;
    std::vector<SegDesc> segs;
    for (auto& kv : classes) {
        uint64_t item = 0;
        const size_t first = segs.size();
        for (size_t i : kv.second) {
            Request* r = act[i];
            SegDesc d{};
            d.item_start = (int64_t)item;
            d.chunk0 = r->next_chunk;
            d.chunk_end = r->next_chunk + grant[i];
            d.col_off = r->arena_off / (r->field == PERMX_FIELD_MODP ? 4 : 8);
            if (r->field == PERMX_FIELD_MODP) {
                d.out_off = (r->arena_off + (int64_t)r->col_bytes) / 8;
                d.p = r->p;
                d.pinv = inv_mod_2_32(r->p);
            } else {
                d.out_off = (r->arena_off + (int64_t)r->col_bytes) / (8 * fp_slot_doubles(r->x64, r->field == PERMX_FIELD_C128));
            }
            segs.push_back(d);
            item += grant[i];
        }
        launches.push_back(L{kv.first.first, kv.first.second, first, (int)(segs.size() - first), item,
                             act[kv.second[0]]});
    }
    double scheduled = 0.0;
    std::vector<Request*> fin;
    for (size_t i = 0; i < act.size(); ++i) {
        scheduled += act[i]->cost * (double)grant[i] / (double)act[i]->chunks;
        act[i]->next_chunk += grant[i];
        if (act[i]->next_chunk == act[i]->chunks && !act[i]->finalizing) fin.push_back(act[i]);
    }
    std::vector<ModpFinalAt> fm;
    std::vector<FpFinal> fc, ff;
    std::vector<Request*> om, oc, of;
    for (Request* r : fin) {
        r->finalizing = true;
        if (r->field == PERMX_FIELD_MODP) {
            ModpFinalAt x{};
            x.acc_index = (r->arena_off + (int64_t)r->col_bytes) / 8;
            x.out_index = (int64_t)fm.size();
            x.p = r->p;
            x.rfix = pow_mod((uint32_t)((1ull << 32) % r->p), (uint64_t)(r->n - 1), r->p);
            x.rfix = (uint32_t)((uint64_t)x.rfix * 2 % r->p);   // Nijenhuis-Wilf factor 2
            x.negate = !(r->n & 1);                             // and sign (-1)^(n-1)
            fm.push_back(x);
            om.push_back(r);
        } else {
            const int pw = fp_slot_doubles(r->x64, r->field == PERMX_FIELD_C128);
            FpFinal x{};
            x.first = (r->arena_off + (int64_t)r->col_bytes) / (8 * pw);
            x.count = (int64_t)(r->chunks >> r->lg);
            x.negate = !(r->n & 1);
            x.twice = 1;
            if (r->field == PERMX_FIELD_C128) {
                x.out_index = (int64_t)fc.size();
                fc.push_back(x);
                oc.push_back(r);
            } else {
                x.out_index = (int64_t)ff.size();
                ff.push_back(x);
                of.push_back(r);
            }
        }
    }
    // layout of the step's metadata buffer
    size_t o_sd[3], o_sx[2], o = 0;
    for (int f = 0; f < 3; ++f) { o_sd[f] = o; o += align256(sd[f].size() * sizeof(StageDesc)); }
    for (int f = 0; f < 2; ++f) { o_sx[f] = o; o += align256(sx[f].size() * sizeof(StageDesc)); }
    const size_t o_seg = o;
    o += align256(segs.size() * sizeof(SegDesc));
    const size_t o_fm = o;
    o += align256(fm.size() * sizeof(ModpFinalAt));
    const size_t o_fc = o;
    o += align256(fc.size() * sizeof(FpFinal));
    const size_t o_ff = o;
    o += align256(ff.size() * sizeof(FpFinal));
    const size_t o_res = o, r_c = 0, r_f = align256(16 * oc.size()), r_m = r_f + align256(8 * of.size());
    const size_t total = o_res + r_m + align256(4 * om.size()) + 256;

    int rc = grow_pinned(&B.h_meta, &B.h_meta_cap, total);
    if (!rc) rc = grow_device(&B.d_meta, &B.d_meta_cap, total);
    if (!rc && up) rc = grow_pinned(&B.h_upload, &B.h_upload_cap, up);
    if (!rc && up) rc = grow_device(&B.d_upload, &B.d_upload_cap, up);
    if (rc) return rc;
    for (int f = 0; f < 3; ++f)
        if (!sd[f].empty()) std::memcpy(B.h_meta + o_sd[f], sd[f].data(), sd[f].size() * sizeof(StageDesc));
    for (int f = 0; f < 2; ++f)
        if (!sx[f].empty()) std::memcpy(B.h_meta + o_sx[f], sx[f].data(), sx[f].size() * sizeof(StageDesc));
    if (!segs.empty()) std::memcpy(B.h_meta + o_seg, segs.data(), segs.size() * sizeof(SegDesc));
    if (!fm.empty()) std::memcpy(B.h_meta + o_fm, fm.data(), fm.size() * sizeof(ModpFinalAt));
    if (!fc.empty()) std::memcpy(B.h_meta + o_fc, fc.data(), fc.size() * sizeof(FpFinal));
    if (!ff.empty()) std::memcpy(B.h_meta + o_ff, ff.data(), ff.size() * sizeof(FpFinal));
    {
        size_t uo = 0;
        for (Request* r : admitted) {
            std::memcpy(B.h_upload + uo, r->host.data(), r->host.size());
            uo += align256(r->host.size());
        }
    }

    // ---- enqueue -------------------------------------------------------------------------
    PERMX_CUDA(cudaEventRecord(B.ev_start, st));
    if (o_res) PERMX_CUDA(cudaMemcpyAsync(B.d_meta, B.h_meta, o_res, cudaMemcpyHostToDevice, st));
    if (up) {
        PERMX_CUDA(cudaMemcpyAsync(B.d_upload, B.h_upload, up, cudaMemcpyHostToDevice, st));
        for (int f = 0; f < 3; ++f) {
            if (sd[f].empty()) continue;
            PERMX_CUDA(launch_stage(f, B.d_upload, reinterpret_cast<const StageDesc*>(B.d_meta + o_sd[f]),
                                    (int64_t)sd[f].size(), S->arena_base, st));
            ++S->launches;
        }
        for (int f = 0; f < 2; ++f) {
            if (sx[f].empty()) continue;
            PERMX_CUDA(launch_stage_x64(f == 0, B.d_upload, reinterpret_cast<const StageDesc*>(B.d_meta + o_sx[f]),
                                        (int64_t)sx[f].size(), S->arena_base, st));
            ++S->launches;
        }
        // F_p accumulators start at zero
        for (Request* r : admitted)
            if (r->field == PERMX_FIELD_MODP)
                PERMX_CUDA(cudaMemsetAsync(S->arena_base + r->arena_off + r->col_bytes, 0, 8, st));
    }
    // classes run on side streams so that small and large classes overlap
    if (!launches.empty()) {
        PERMX_CUDA(cudaEventRecord(S->ev_ready[slot], st));
        const int used = std::min<int>((int)launches.size(), kSideStreams);
        for (int q = 0; q < used; ++q) PERMX_CUDA(cudaStreamWaitEvent(S->side[q], S->ev_ready[slot], 0));
        int li = 0;
        for (const L& l : launches) {
            cudaStream_t ls = S->side[li++ % kSideStreams];
            const SegDesc* sg = reinterpret_cast<const SegDesc*>(B.d_meta + o_seg) + l.off;
            cudaError_t e;
            if (l.field == PERMX_FIELD_MODP) {
                ModpLaunch M;
                M.colT = reinterpret_cast<const uint32_t*>(S->arena_base);
                M.p = M.pinv = nullptr;
                M.acc = reinterpret_cast<unsigned long long*>(S->arena_base);
                M.mat_stride = 0;
                M.item_begin = 0;
                M.item_end = l.items;
                M.k_lo = 0;
                M.k_hi = ~0ull;
                M.ell = l.any->ell;
                M.log2_chunks = l.any->log2_chunks;
                M.segs = sg;
                M.nsegs = l.nseg;
                M.nw = 1;
                e = dispatch_modp(l.n, M, ls);
            } else {
                FpLaunch F;
                F.colT = reinterpret_cast<const double*>(S->arena_base);
                F.partial = reinterpret_cast<double*>(S->arena_base);
                F.mat_stride = 0;
                F.item_begin = 0;
                F.item_end = l.items;
                F.ell = l.any->ell;
                F.log2_chunks = l.any->log2_chunks;
                F.segs = sg;
                F.nsegs = l.nseg;
                F.nw = 1;
                if (l.any->x64) e = l.field == PERMX_FIELD_C128 ? dispatch_x64c(l.n, F, ls) : dispatch_x64r(l.n, F, ls);
                else e = l.field == PERMX_FIELD_C128 ? dispatch_c128(l.n, F, ls) : dispatch_f64(l.n, F, ls);
            }
            if (e != cudaSuccess) return cuda_fail(e, "server step launch");
            ++S->launches;
        }
        for (int q = 0; q < used; ++q) {
            PERMX_CUDA(cudaEventRecord(S->ev_side[slot][q], S->side[q]));
            PERMX_CUDA(cudaStreamWaitEvent(st, S->ev_side[slot][q], 0));
        }
    }
    // ---- finalise the requests whose last chunk ran in this step ---------------------------
    if (!fin.empty()) {
        unsigned char* dres = B.d_meta + o_res;
        PERMX_CUDA(launch_finalize_modp_at(reinterpret_cast<const unsigned long long*>(S->arena_base),
                                           reinterpret_cast<const ModpFinalAt*>(B.d_meta + o_fm), (int64_t)fm.size(),
                                           reinterpret_cast<uint32_t*>(dres + r_m), st));
        PERMX_CUDA(launch_finalize_fp(reinterpret_cast<const double*>(S->arena_base),
                                      reinterpret_cast<const FpFinal*>(B.d_meta + o_fc), (int64_t)fc.size(), true,
                                      S->x64, dres + r_c, st));
        PERMX_CUDA(launch_finalize_fp(reinterpret_cast<const double*>(S->arena_base),
                                      reinterpret_cast<const FpFinal*>(B.d_meta + o_ff), (int64_t)ff.size(), false,
                                      S->x64, dres + r_f, st));
        S->launches += (!fm.empty()) + (!fc.empty()) + (!ff.empty());
        PERMX_CUDA(cudaMemcpyAsync(B.h_meta + o_res, dres, total - 256 - o_res, cudaMemcpyDeviceToHost, st));
        for (size_t i = 0; i < oc.size(); ++i) B.results.push_back({oc[i], o_res + r_c + 16 * i});
        for (size_t i = 0; i < of.size(); ++i) B.results.push_back({of[i], o_res + r_f + 8 * i});
        for (size_t i = 0; i < om.size(); ++i) B.results.push_back({om[i], o_res + r_m + 4 * i});
    }
    PERMX_CUDA(cudaEventRecord(B.ev_end, st));
    B.busy = true;
    B.work = scheduled;
    ++S->steps;
    return PERMX_OK;
}

// Wait for a step, then hand its finished requests their results.
int reap_step(perm_server* S, StepBuf& B) {
    if (!B.busy) return PERMX_OK;
    B.busy = false;
    PERMX_CUDA(cudaEventSynchronize(B.ev_end));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, B.ev_start, B.ev_end) != cudaSuccess) ms = 0.f;
    const int64_t t = now_ns();
    for (auto& rr : B.results) std::memcpy(rr.first->result, B.h_meta + rr.second, entry_bytes(rr.first->field));
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->gpu_busy_ms += ms;
        S->resident_work = std::max(0.0, S->resident_work - B.work);
        for (auto& rr : B.results) {
            Request* r = rr.first;
            r->done = true;
            r->t_done = t;
            r->host.clear();
            r->host.shrink_to_fit();
            S->arena.release((size_t)r->arena_off, r->bytes);
            S->resident.erase(std::find(S->resident.begin(), S->resident.end(), r));
            ++S->completed;
        }
    }
    B.results.clear();
    S->cv_done.notify_all();
    return PERMX_OK;
}

// baseline: one request, one batched call of one matrix
int run_plain(perm_server* S, Request* r) {
    cudaStream_t st = S->stream;
    int rc = grow_device(&S->d_plain, &S->d_plain_cap, align256(r->host.size()) + 256);
    if (rc) return rc;
    cudaEvent_t e0 = S->buf[0].ev_start, e1 = S->buf[0].ev_end;
    PERMX_CUDA(cudaEventRecord(e0, st));
    PERMX_CUDA(cudaMemcpyAsync(S->d_plain, r->host.data(), r->host.size(), cudaMemcpyHostToDevice, st));
    unsigned char* out = S->d_plain + align256(r->host.size());
    const int32_t n = r->n;
    const int64_t off = 0;
    if (r->field == PERMX_FIELD_MODP)
        rc = run_modp_batch(reinterpret_cast<const uint32_t*>(S->d_plain), &n, &off, &r->p, 1,
                            reinterpret_cast<uint32_t*>(out), st);
    else
        rc = run_fp_batch(reinterpret_cast<const double*>(S->d_plain), &n, &off, 1, out,
                          r->field == PERMX_FIELD_C128, st);
    if (rc) return rc;
    PERMX_CUDA(cudaMemcpyAsync(r->result, out, entry_bytes(r->field), cudaMemcpyDeviceToHost, st));
    PERMX_CUDA(cudaEventRecord(e1, st));
    PERMX_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 0.f;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->done = true;
        r->t_done = now_ns();
        r->host.clear();
        S->launches += 3;
        S->gpu_busy_ms += ms;
        ++S->completed;
        ++S->steps;
    }
    S->cv_done.notify_all();
    return PERMX_OK;
}

void worker_main(perm_server* S) {
    cudaSetDevice(S->cfg.device);
    uint64_t k = 0;   // steps enqueued; step k uses buffer set k & 1
    int rc = PERMX_OK;
    while (rc == PERMX_OK) {
        std::vector<Request*> admitted;
        Request* plain = nullptr;
        bool work = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            const bool inflight = S->buf[0].busy || S->buf[1].busy;
            if (!inflight)
                S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty() || has_grantable(S); });
            if (S->stop) break;
            if (S->cfg.plain_fifo) {
                if (!S->pending.empty()) {
                    plain = S->pending.front();
                    S->pending.pop_front();
                }
            } else {
                admit(S, admitted);
                work = has_grantable(S);
            }
        }
        if (plain) {
            rc = run_plain(S, plain);
        } else if (work) {
            StepBuf& B = S->buf[k & 1];
            rc = reap_step(S, B);   // the step that used this buffer set two steps ago
            if (rc == PERMX_OK) rc = enqueue_step(S, B, (int)(k & 1), admitted);
            ++k;
        } else {
            // nothing to schedule: wait for the older step in flight
            StepBuf& older = S->buf[k & 1].busy ? S->buf[k & 1] : S->buf[(k + 1) & 1];
            rc = reap_step(S, older);
        }
        // results of steps that have already completed
        for (int q = 0; q < 2 && rc == PERMX_OK; ++q) {
            StepBuf& B = S->buf[(k + q) & 1];   // older first
            if (B.busy && cudaEventQuery(B.ev_end) == cudaSuccess) rc = reap_step(S, B);
            else break;
        }
    }
    if (rc) {
        // a failed step leaves the device state unknown: stop serving
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->worker_error) {
            S->worker_error = rc;
            S->worker_msg = perm_last_error();
        }
        S->stop = true;
    }
    S->cv_done.notify_all();
}

void destroy_buffers(perm_server* S) {
    for (StepBuf& B : S->buf) {
        if (B.d_meta) cudaFree(B.d_meta);
        if (B.d_upload) cudaFree(B.d_upload);
        if (B.h_meta) cudaFreeHost(B.h_meta);
        if (B.h_upload) cudaFreeHost(B.h_upload);
        if (B.ev_start) cudaEventDestroy(B.ev_start);
        if (B.ev_end) cudaEventDestroy(B.ev_end);
        B = StepBuf{};
    }
    for (int s = 0; s < 2; ++s) {
        if (S->ev_ready[s]) cudaEventDestroy(S->ev_ready[s]);
        for (int q = 0; q < kSideStreams; ++q)
            if (S->ev_side[s][q]) cudaEventDestroy(S->ev_side[s][q]);
    }
    for (int q = 0; q < kSideStreams; ++q)
        if (S->side[q]) cudaStreamDestroy(S->side[q]);
    if (S->d_plain) cudaFree(S->d_plain);
    if (S->arena_base) cudaFree(S->arena_base);
    if (S->stream) cudaStreamDestroy(S->stream);
}

}  // namespace

extern "C" {

int serve_create(const perm_serve_cfg* cfg, perm_server** h) {
    clear_error();
    if (!h) return fail(PERMX_EINVAL, "NULL handle pointer");
    perm_server* S = new perm_server();
    if (cfg) S->cfg = *cfg;
    if (S->cfg.max_requests <= 0) S->cfg.max_requests = 65536;
    if (S->cfg.max_resident <= 0) S->cfg.max_resident = 4096;
    if (S->cfg.device_bytes <= 0) S->cfg.device_bytes = (int64_t)1 << 30;
    if (S->cfg.chunks_per_step < 0) S->cfg.chunks_per_step = 0;
    if (S->cfg.work_budget == 0) S->cfg.work_budget = kDefaultWorkBudget;
    cudaError_t e = cudaSetDevice(S->cfg.device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    for (int q = 0; q < kSideStreams && e == cudaSuccess; ++q)
        e = cudaStreamCreateWithFlags(&S->side[q], cudaStreamNonBlocking);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
        e = cudaEventCreateWithFlags(&S->ev_ready[s], cudaEventDisableTiming);
        for (int q = 0; q < kSideStreams && e == cudaSuccess; ++q)
            e = cudaEventCreateWithFlags(&S->ev_side[s][q], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&S->buf[s].ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&S->buf[s].ev_end);
    }
    if (e == cudaSuccess && !S->cfg.plain_fifo)
        e = cudaMalloc(reinterpret_cast<void**>(&S->arena_base), (size_t)S->cfg.device_bytes);
    if (e != cudaSuccess) {
        destroy_buffers(S);
        delete S;
        return cuda_fail(e, "serve_create");
    }
    S->arena.reset(S->cfg.plain_fifo ? 0 : (size_t)S->cfg.device_bytes);
    S->x64 = fp_arith() == 1;
    S->t_create = now_ns();
    S->worker = std::thread(worker_main, S);
    *h = S;
    return PERMX_OK;
}

int serve_submit(perm_server* S, int field, int32_t n, const void* A_host, uint32_t p, uint64_t* ticket) {
    clear_error();
    if (!S || !A_host || !ticket) return fail(PERMX_EINVAL, "NULL argument");
    if (field != PERMX_FIELD_C128 && field != PERMX_FIELD_F64 && field != PERMX_FIELD_MODP)
        return fail(PERMX_EINVAL, "unknown field");
    const int maxn = field == PERMX_FIELD_MODP ? PERMX_MAX_N_MODP : PERMX_MAX_N_FP;
    if (n < 1 || n > maxn) return fail(PERMX_EINVAL, "n out of range");
    if (field == PERMX_FIELD_MODP) {
        if (p <= 2 || p >= (1u << 31) || !is_prime_u32(p)) return fail(PERMX_EINVAL, "p is not an odd prime below 2^31");
        const uint32_t* a = static_cast<const uint32_t*>(A_host);
        for (int64_t e = 0; e < (int64_t)n * n; ++e)
            if (a[e] >= p) return fail(PERMX_EINVAL, "entry >= p");
    }
    Request* r = new Request();
    r->field = field;
    r->n = n;
    r->p = p;
    const size_t bytes = (size_t)n * n * entry_bytes(field);
    r->host.assign(static_cast<const unsigned char*>(A_host), static_cast<const unsigned char*>(A_host) + bytes);
    plan_request(r, S->x64);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->worker_error) {
            delete r;
            return fail(S->worker_error, "server stopped after an error: " + S->worker_msg);
        }
        if ((int64_t)S->live.size() >= S->cfg.max_requests) {
            delete r;
            return fail(PERMX_EBUSY, "request capacity reached; poll finished tickets first");
        }
        if (!S->cfg.plain_fifo && r->bytes > (size_t)S->cfg.device_bytes) {
            delete r;
            return fail(PERMX_EINVAL, "request larger than the server's device budget");
        }
        r->ticket = S->next_ticket++;
        r->t_submit = now_ns();
        S->live[r->ticket] = r;
        S->pending.push_back(r);
        ++S->submitted;
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return PERMX_OK;
}

int serve_poll_timed(perm_server* S, uint64_t ticket, void* result, int* done, int64_t* t_submit_ns,
                     int64_t* t_done_ns) {
    clear_error();
    if (!S || !done) return fail(PERMX_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) {
        if (S->worker_error) return fail(S->worker_error, "server stopped after an error: " + S->worker_msg);
        return fail(PERMX_ENOTFOUND, "unknown ticket");
    }
    Request* r = it->second;
    if (!r->done) {
        *done = 0;
        if (S->worker_error) return fail(S->worker_error, "server stopped after an error: " + S->worker_msg);
        return PERMX_OK;
    }
    *done = 1;
    if (result) std::memcpy(result, r->result, entry_bytes(r->field));
    if (t_submit_ns) *t_submit_ns = r->t_submit;
    if (t_done_ns) *t_done_ns = r->t_done;
    S->live.erase(it);
    delete r;
    return PERMX_OK;
}

int serve_poll(perm_server* S, uint64_t ticket, void* result, int* done) {
    return serve_poll_timed(S, ticket, result, done, nullptr, nullptr);
}

int serve_drain(perm_server* S, int64_t timeout_ms) {
    clear_error();
    if (!S) return fail(PERMX_EINVAL, "NULL handle");
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return S->completed == S->submitted || S->worker_error; });
    if (S->worker_error) return fail(S->worker_error, "server stopped after an error: " + S->worker_msg);
    if (!ok) return fail(PERMX_ETIMEOUT, "requests still in flight");
    return PERMX_OK;
}

int serve_stats(perm_server* S, int64_t* stats5) {
    clear_error();
    if (!S || !stats5) return fail(PERMX_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    stats5[0] = S->submitted;
    stats5[1] = S->completed;
    stats5[2] = (int64_t)S->resident.size();
    stats5[3] = S->steps;
    stats5[4] = S->launches;
    return PERMX_OK;
}

int serve_stats2(perm_server* S, perm_serve_stats* out) {
    clear_error();
    if (!S || !out) return fail(PERMX_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->resident = (int64_t)S->resident.size();
    out->steps = S->steps;
    out->launches = S->launches;
    out->pending = (int64_t)S->pending.size();
    out->resident_work = (int64_t)S->resident_work;
    out->gpu_busy_ms = S->gpu_busy_ms;
    out->uptime_ms = (double)(now_ns() - S->t_create) * 1e-6;
    return PERMX_OK;
}

int serve_destroy(perm_server* S) {
    clear_error();
    if (!S) return fail(PERMX_EINVAL, "NULL handle");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->cfg.device);
    cudaStreamSynchronize(S->stream);
    for (int q = 0; q < kSideStreams; ++q)
        if (S->side[q]) cudaStreamSynchronize(S->side[q]);
    for (auto& kv : S->live) delete kv.second;
    destroy_buffers(S);
    delete S;
    return PERMX_OK;
}

}  // extern "C"
