// Serving: continuous batching of permanent requests (include/permx.h,
// serve_*).  A worker thread runs steps.  Each step
//   1. admits queued requests while resident slots and the device-memory
//      arena allow (admission by memory and by count),
//   2. stages the newly admitted matrices column-major in the arena,
//   3. grants every resident request a share of the step's work budget in
//      whole lane groups of Gray-code chunks (oldest first, every request at
//      least one group) and launches one segment-mode Ryser kernel per
//      (field, n) class present,
//   4. finalises the requests whose last chunk ran and copies their results
//      back.
// Requests that arrive while a step runs join at the next step.  A request is
// cut into exactly the chunks and lane groups of the batched path and its
// partial slots are summed by the same fixed-order finalize kernel, so its
// result is bit-identical to perm_c128 / perm_f64 / perm_modp on that matrix.
//
// plain_fifo = 1 is the baseline: one request at a time, each as its own
// batched call of one matrix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
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
    int64_t arena_off = -1;            // columns, then partial slots / accumulator
    size_t bytes = 0, col_bytes = 0;
    bool done = false;
    unsigned char result[16] = {0};
    int64_t t_submit = 0, t_done = 0;
};

int entry_bytes(int field) { return field == PERMX_FIELD_C128 ? 16 : field == PERMX_FIELD_F64 ? 8 : 4; }


}  // namespace
}  // namespace permx

using namespace permx;

constexpr int kSideStreams = 4;

struct perm_server {
    perm_serve_cfg cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t side[kSideStreams] = {nullptr};
    cudaEvent_t ev_ready = nullptr, ev_side[kSideStreams] = {nullptr};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<Request*> pending;
    std::vector<Request*> resident;
    std::unordered_map<uint64_t, Request*> live;   // every ticket not yet reported done by a poll
    int64_t submitted = 0, completed = 0;
    std::atomic<int64_t> steps{0}, launches{0};
    int worker_error = 0;
    bool x64 = true;                   // float arithmetic fixed when the server is created
    std::string worker_msg;
    // device / pinned buffers owned by the worker
    unsigned char* arena_base = nullptr;
    Arena arena;
    unsigned char* d_meta = nullptr;
    size_t d_meta_cap = 0;
    unsigned char* h_meta = nullptr;
    size_t h_meta_cap = 0;
    unsigned char* d_upload = nullptr;
    size_t d_upload_cap = 0;
    unsigned char* h_upload = nullptr;
    size_t h_upload_cap = 0;
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
    const size_t tail = modp ? 8 : (size_t)(r->chunks >> r->lg) * (r->field == PERMX_FIELD_C128 ? 32 : 16);
    r->bytes = r->col_bytes + align256(tail);
}

// one step of the continuous-batching loop; returns PERMX_OK or an error code
int run_step(perm_server* S, std::vector<Request*>& admitted) {
    cudaStream_t st = S->stream;
    // ---- stage newly admitted matrices ------------------------------------------------
    if (!admitted.empty()) {
        size_t up = 0;
        for (Request* r : admitted) up += align256(r->host.size());
        int rc = grow_pinned(&S->h_upload, &S->h_upload_cap, up);
        if (!rc) rc = grow_device(&S->d_upload, &S->d_upload_cap, up);
        if (rc) return rc;
        std::vector<StageDesc> sd[3], sx[2];   // sx: integer-mantissa staging [complex, real]
        size_t o = 0;
        for (Request* r : admitted) {
            std::memcpy(S->h_upload + o, r->host.data(), r->host.size());
            const int eb = entry_bytes(r->field);
            const StageDesc d{(int64_t)(o / eb), (int64_t)(r->arena_off / eb), r->n, r->ld, r->p, 1};
            if (r->x64) sx[r->field == PERMX_FIELD_C128 ? 0 : 1].push_back(d);
            else sd[r->field].push_back(d);
            o += align256(r->host.size());
        }
        PERMX_CUDA(cudaMemcpyAsync(S->d_upload, S->h_upload, up, cudaMemcpyHostToDevice, st));
        size_t meta = 0;
        for (auto& v : sd) meta += align256(v.size() * sizeof(StageDesc));
        for (auto& v : sx) meta += align256(v.size() * sizeof(StageDesc));
        rc = grow_pinned(&S->h_meta, &S->h_meta_cap, meta);
        if (!rc) rc = grow_device(&S->d_meta, &S->d_meta_cap, meta);
        if (rc) return rc;
        size_t mo = 0;
        for (int f = 0; f < 3; ++f) {
            if (sd[f].empty()) continue;
            std::memcpy(S->h_meta + mo, sd[f].data(), sd[f].size() * sizeof(StageDesc));
            mo += align256(sd[f].size() * sizeof(StageDesc));
        }
        for (int f = 0; f < 2; ++f) {
            if (sx[f].empty()) continue;
            std::memcpy(S->h_meta + mo, sx[f].data(), sx[f].size() * sizeof(StageDesc));
            mo += align256(sx[f].size() * sizeof(StageDesc));
        }
        PERMX_CUDA(cudaMemcpyAsync(S->d_meta, S->h_meta, mo, cudaMemcpyHostToDevice, st));
        mo = 0;
        for (int f = 0; f < 3; ++f) {
            if (sd[f].empty()) continue;
            PERMX_CUDA(launch_stage(f, S->d_upload, reinterpret_cast<const StageDesc*>(S->d_meta + mo),
                                    (int64_t)sd[f].size(), S->arena_base, st));
            ++S->launches;
            mo += align256(sd[f].size() * sizeof(StageDesc));
        }
        for (int f = 0; f < 2; ++f) {
            if (sx[f].empty()) continue;
            PERMX_CUDA(launch_stage_x64(f == 0, S->d_upload, reinterpret_cast<const StageDesc*>(S->d_meta + mo),
                                        (int64_t)sx[f].size(), S->arena_base, st));
            ++S->launches;
            mo += align256(sx[f].size() * sizeof(StageDesc));
        }
        // F_p accumulators start at zero
        for (Request* r : admitted)
            if (r->field == PERMX_FIELD_MODP)
                PERMX_CUDA(cudaMemsetAsync(S->arena_base + r->arena_off + r->col_bytes, 0, 8, st));
        // the metadata buffer is reused below: wait for the staging to read it
        PERMX_CUDA(cudaStreamSynchronize(st));
    }

    // ---- grant work ----------------------------------------------------------------------
    // A chunk is one thread's Gray walk.  Per step every (field, n) class may
    // run one wave of its kernel's resident threads (classes run concurrently
    // on the side streams), or chunks_per_step chunks in total when set.
    // Within a class every request first gets a fair share (at least one lane
    // group), then the rest of the wave goes to the oldest requests first.
    std::vector<Request*> act = S->resident;   // admission order
    std::vector<uint64_t> grant(act.size(), 0);
    std::map<std::pair<int, int>, std::vector<size_t>> by_class;
    for (size_t i = 0; i < act.size(); ++i) by_class[{act[i]->field, act[i]->n}].push_back(i);
    const int64_t fixed = S->cfg.chunks_per_step;
    for (auto& kv : by_class) {
        const std::vector<size_t>& idx = kv.second;
        Request* r0 = act[idx[0]];
        const int kind = r0->field == PERMX_FIELD_MODP ? 0
                         : r0->field == PERMX_FIELD_F64 ? (r0->x64 ? 3 : 1) : (r0->x64 ? 4 : 2);
        int64_t budget = fixed > 0 ? std::max<int64_t>(1, fixed / (int64_t)by_class.size())
                                   : (int64_t)sm_count() * dispatch_blocks_per_sm(kind, r0->n) * kRyserThreads;
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
    // ---- segment tables, one launch per (field, n) ------------------------------------------
    std::map<std::pair<int, int>, std::vector<size_t>> classes;
    for (size_t i = 0; i < act.size(); ++i)
        if (grant[i]) classes[{act[i]->field, act[i]->n}].push_back(i);
    size_t meta = 0;
    for (auto& kv : classes) meta += align256(kv.second.size() * sizeof(SegDesc));
    int rc = grow_pinned(&S->h_meta, &S->h_meta_cap, meta + 256);
    if (!rc) rc = grow_device(&S->d_meta, &S->d_meta_cap, meta + 256);
    if (rc) return rc;
    size_t mo = 0;
    struct L { int field, n; size_t off; int nseg; uint64_t items; Request* any; };
    std::vector<L> launches;
    for (auto& kv : classes) {
        SegDesc* sd = reinterpret_cast<SegDesc*>(S->h_meta + mo);
        uint64_t item = 0;
        int k = 0;
        for (size_t i : kv.second) {
            Request* r = act[i];
            SegDesc d{};
            d.item_start = (int64_t)item;
            d.chunk0 = r->next_chunk;
            d.chunk_end = r->next_chunk + grant[i];
            const int eb = entry_bytes(r->field);
            d.col_off = r->arena_off / (r->field == PERMX_FIELD_MODP ? 4 : 8);
            (void)eb;
            if (r->field == PERMX_FIELD_MODP) {
                d.out_off = (r->arena_off + (int64_t)r->col_bytes) / 8;
                d.p = r->p;
                d.pinv = inv_mod_2_32(r->p);
            } else {
                d.out_off = (r->arena_off + (int64_t)r->col_bytes) / (r->field == PERMX_FIELD_C128 ? 32 : 16);
            }
            sd[k++] = d;
            item += grant[i];
        }
        launches.push_back(L{kv.first.first, kv.first.second, mo, k, item, act[kv.second[0]]});
        mo += align256(kv.second.size() * sizeof(SegDesc));
    }
    if (mo) PERMX_CUDA(cudaMemcpyAsync(S->d_meta, S->h_meta, mo, cudaMemcpyHostToDevice, st));
    // classes run on side streams so that small and large classes overlap
    PERMX_CUDA(cudaEventRecord(S->ev_ready, st));
    for (int q = 0; q < kSideStreams; ++q) PERMX_CUDA(cudaStreamWaitEvent(S->side[q], S->ev_ready, 0));
    int li = 0;
    for (const L& l : launches) {
        cudaStream_t ls = S->side[li++ % kSideStreams];
        const SegDesc* segs = reinterpret_cast<const SegDesc*>(S->d_meta + l.off);
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
            M.segs = segs;
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
            F.segs = segs;
            F.nsegs = l.nseg;
            F.nw = 1;
            if (l.any->x64) e = l.field == PERMX_FIELD_C128 ? dispatch_x64c(l.n, F, ls) : dispatch_x64r(l.n, F, ls);
            else e = l.field == PERMX_FIELD_C128 ? dispatch_c128(l.n, F, ls) : dispatch_f64(l.n, F, ls);
        }
        if (e != cudaSuccess) return cuda_fail(e, "server step launch");
        ++S->launches;
    }
    for (int q = 0; q < kSideStreams; ++q) {
        PERMX_CUDA(cudaEventRecord(S->ev_side[q], S->side[q]));
        PERMX_CUDA(cudaStreamWaitEvent(st, S->ev_side[q], 0));
    }
    for (size_t i = 0; i < act.size(); ++i) act[i]->next_chunk += grant[i];

    // ---- finalise finished requests ---------------------------------------------------------
    std::vector<Request*> fin;
    for (Request* r : act)
        if (r->next_chunk == r->chunks) fin.push_back(r);
    if (!fin.empty()) {
        std::vector<ModpFinalAt> fm;
        std::vector<FpFinal> fc, ff;
        std::vector<Request*> om, oc, of;
        for (Request* r : fin) {
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
                const int pw = r->field == PERMX_FIELD_C128 ? 4 : 2;
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
        // results: [c128 x16][f64 x8][modp x4]
        const size_t o_fm = align256(mo), o_fc = o_fm + align256(fm.size() * sizeof(ModpFinalAt));
        const size_t o_ff = o_fc + align256(fc.size() * sizeof(FpFinal));
        const size_t o_res = o_ff + align256(ff.size() * sizeof(FpFinal));
        const size_t r_c = 0, r_f = align256(16 * oc.size()), r_m = r_f + align256(8 * of.size());
        const size_t total = o_res + r_m + align256(4 * om.size());
        if (S->h_meta_cap < total || S->d_meta_cap < total) {
            // the segment tables in the device buffer are still in use by queued kernels
            // the pinned and device metadata are still read by queued copies and kernels
            PERMX_CUDA(cudaStreamSynchronize(st));
            rc = grow_pinned(&S->h_meta, &S->h_meta_cap, total);
            if (!rc) rc = grow_device(&S->d_meta, &S->d_meta_cap, total);
            if (rc) return rc;
            // the segment tables were consumed; nothing else lives below o_fm
        }
        std::memcpy(S->h_meta + o_fm, fm.data(), fm.size() * sizeof(ModpFinalAt));
        std::memcpy(S->h_meta + o_fc, fc.data(), fc.size() * sizeof(FpFinal));
        std::memcpy(S->h_meta + o_ff, ff.data(), ff.size() * sizeof(FpFinal));
        PERMX_CUDA(cudaMemcpyAsync(S->d_meta + o_fm, S->h_meta + o_fm, o_res - o_fm, cudaMemcpyHostToDevice, st));
        unsigned char* dres = S->d_meta + o_res;
        PERMX_CUDA(launch_finalize_modp_at(reinterpret_cast<const unsigned long long*>(S->arena_base),
                                           reinterpret_cast<const ModpFinalAt*>(S->d_meta + o_fm),
                                           (int64_t)fm.size(), reinterpret_cast<uint32_t*>(dres + r_m), st));
        PERMX_CUDA(launch_finalize_fp(reinterpret_cast<const double*>(S->arena_base),
                                      reinterpret_cast<const FpFinal*>(S->d_meta + o_fc), (int64_t)fc.size(), true,
                                      dres + r_c, st));
        PERMX_CUDA(launch_finalize_fp(reinterpret_cast<const double*>(S->arena_base),
                                      reinterpret_cast<const FpFinal*>(S->d_meta + o_ff), (int64_t)ff.size(), false,
                                      dres + r_f, st));
        S->launches += (!fm.empty()) + (!fc.empty()) + (!ff.empty());
        PERMX_CUDA(cudaMemcpyAsync(S->h_meta + o_res, dres, total - o_res, cudaMemcpyDeviceToHost, st));
        PERMX_CUDA(cudaStreamSynchronize(st));
        const int64_t t = now_ns();
        for (size_t i = 0; i < oc.size(); ++i) std::memcpy(oc[i]->result, S->h_meta + o_res + r_c + 16 * i, 16);
        for (size_t i = 0; i < of.size(); ++i) std::memcpy(of[i]->result, S->h_meta + o_res + r_f + 8 * i, 8);
        for (size_t i = 0; i < om.size(); ++i) std::memcpy(om[i]->result, S->h_meta + o_res + r_m + 4 * i, 4);
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request* r : fin) {
            r->done = true;
            r->t_done = t;
            r->host.clear();
            r->host.shrink_to_fit();
            S->arena.release((size_t)r->arena_off, r->bytes);
            S->resident.erase(std::find(S->resident.begin(), S->resident.end(), r));
            ++S->completed;
        }
    } else {
        PERMX_CUDA(cudaStreamSynchronize(st));
    }
    return PERMX_OK;
}

// baseline: one request, one batched call of one matrix
int run_plain(perm_server* S, Request* r) {
    cudaStream_t st = S->stream;
    int rc = grow_device(&S->d_upload, &S->d_upload_cap, align256(r->host.size()) + 256);
    if (rc) return rc;
    PERMX_CUDA(cudaMemcpyAsync(S->d_upload, r->host.data(), r->host.size(), cudaMemcpyHostToDevice, st));
    unsigned char* out = S->d_upload + align256(r->host.size());
    const int32_t n = r->n;
    const int64_t off = 0;
    if (r->field == PERMX_FIELD_MODP)
        rc = run_modp_batch(reinterpret_cast<const uint32_t*>(S->d_upload), &n, &off, &r->p, 1,
                            reinterpret_cast<uint32_t*>(out), st);
    else
        rc = run_fp_batch(reinterpret_cast<const double*>(S->d_upload), &n, &off, 1, out,
                          r->field == PERMX_FIELD_C128, st);
    if (rc) return rc;
    PERMX_CUDA(cudaMemcpyAsync(r->result, out, entry_bytes(r->field), cudaMemcpyDeviceToHost, st));
    PERMX_CUDA(cudaStreamSynchronize(st));
    std::lock_guard<std::mutex> lk(S->mu);
    r->done = true;
    r->t_done = now_ns();
    r->host.clear();
    S->launches += 3;
    ++S->completed;
    ++S->steps;
    return PERMX_OK;
}

void worker_main(perm_server* S) {
    cudaSetDevice(S->cfg.device);
    while (true) {
        std::vector<Request*> admitted;
        Request* plain = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->resident.empty(); });
            if (S->stop) return;
            if (S->cfg.plain_fifo) {
                plain = S->pending.front();
                S->pending.pop_front();
            } else {
                while (!S->pending.empty() && (int64_t)S->resident.size() < S->cfg.max_resident) {
                    Request* r = S->pending.front();
                    const int64_t off = S->arena.alloc(r->bytes);
                    if (off < 0) break;   // memory-bound admission: wait for residents to finish
                    r->arena_off = off;
                    S->pending.pop_front();
                    S->resident.push_back(r);
                    admitted.push_back(r);
                }
            }
        }
        int rc = plain ? run_plain(S, plain) : run_step(S, admitted);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (!plain) ++S->steps;
            if (rc && !S->worker_error) {
                S->worker_error = rc;
                S->worker_msg = perm_last_error();
            }
        }
        S->cv_done.notify_all();
        if (rc) {
            // a failed step leaves the device state unknown: stop serving
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
            return;
        }
    }
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
    cudaError_t e = cudaSetDevice(S->cfg.device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    for (int q = 0; q < kSideStreams && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&S->side[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_side[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_ready, cudaEventDisableTiming);
    if (e == cudaSuccess && !S->cfg.plain_fifo)
        e = cudaMalloc(reinterpret_cast<void**>(&S->arena_base), (size_t)S->cfg.device_bytes);
    if (e != cudaSuccess) {
        if (S->stream) cudaStreamDestroy(S->stream);
        delete S;
        return cuda_fail(e, "serve_create");
    }
    S->arena.reset(S->cfg.plain_fifo ? 0 : (size_t)S->cfg.device_bytes);
    S->x64 = fp_arith() == 1;
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
    for (auto& kv : S->live) delete kv.second;
    if (S->arena_base) cudaFree(S->arena_base);
    if (S->d_meta) cudaFree(S->d_meta);
    if (S->d_upload) cudaFree(S->d_upload);
    if (S->h_meta) cudaFreeHost(S->h_meta);
    if (S->h_upload) cudaFreeHost(S->h_upload);
    for (int q = 0; q < kSideStreams; ++q) {
        if (S->side[q]) cudaStreamDestroy(S->side[q]);
        if (S->ev_side[q]) cudaEventDestroy(S->ev_side[q]);
    }
    if (S->ev_ready) cudaEventDestroy(S->ev_ready);
    cudaStreamDestroy(S->stream);
    delete S;
    return PERMX_OK;
}

}  // extern "C"
