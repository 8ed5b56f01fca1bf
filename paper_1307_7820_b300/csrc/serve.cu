// serve.cu -- continuous-batching serving loop of libfold_b300.
//
// A host scheduler thread owns one device arena of `budget_bytes`.  Submitted
// requests wait in a FIFO until their workspace (D copies, difference
// vectors, tile flags: the single-sequence plan) fits the arena and fewer
// than `max_inflight` requests are in flight.  The thread then folds every
// in-flight request in repeated persistent launches; each launch runs, for
// every request, the tasks of its next kSlice tile diagonals (the same
// ordered task list a single fold uses, cut at step boundaries), so requests
// admitted while others are running join the next launch and share the GPU
// with them.  All in-flight DP state stays in the arena between launches.  A
// finished request keeps its block until its ticket is polled.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "fold.h"
#include "fold_common.h"
#include "kernels.h"
#include "schedule.h"

namespace fold {

constexpr int kSliceMin = 2;         // tile diagonals per request per launch: adapted so that one
constexpr int kSliceMax = 64;        // launch takes about kSliceTargetMs
constexpr double kSliceTargetMs = 2.0;
constexpr size_t kMaxQueued = 1 << 20;

struct Request {
    uint64_t ticket = 0;
    int n = 0;
    int NT = 0;
    std::vector<uint8_t> codes;      // padded to Np with the padding code
    Plan pl;
    size_t block = 0;                // arena byte offset
    size_t bytes = 0;
    std::vector<int4> tasks;
    std::vector<int> step_begin;
    int cursor = 0;                  // next tile diagonal to schedule
    int state = 0;                   // 0 queued, 1 in flight, 2 done, 3 failed
    int status = FOLD_OK;
    int32_t result = 0;
};

// first-fit allocator over [0, size) in 256-byte units
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(size_t s) { size = s; free_.clear(); free_[0] = s; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, o = it->first + bytes;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct ServeState {
    fold_ctx *ctx = nullptr;
    size_t budget = 0;
    int max_inflight = 0;
    uint8_t *arena_base = nullptr;
    Arena arena;
    cudaStream_t st = nullptr;       // scheduler stream
    cudaStream_t poll_st = nullptr;  // extraction of finished tables
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queued;
    std::vector<uint64_t> inflight;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    // launch buffers
    DevBuf d_launch;                 // control | results | SeqDesc | tasks
    HostBuf h_launch;
    unsigned long long launches = 0;
};

static size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// SeqDesc of a request whose plan sits at arena byte offset `block`; every
// pool pointer of the launch is the arena base, so offsets are in elements.
static SeqDesc arena_desc(const Request &r, int slot) {
    SeqDesc d = r.pl.sd[0];
    const size_t B = r.block;
    d.code_off = (long long)(B + r.pl.off_codes);
    d.drow_off = (long long)((B + r.pl.off_drow) / 2);
    d.dcol_off = (long long)((B + r.pl.off_dcol) / 2);
    d.rf_off = (long long)((B + r.pl.off_rf) / 4);
    d.cf_off = (long long)((B + r.pl.off_cf) / 4);
    d.flag_off = (long long)((B + r.pl.off_flags) / 4);
    d.cnt_off = (long long)((B + r.pl.off_cnt) / 4);
    d.p_off = (long long)((B + r.pl.off_pring) / 4);
    d.result_index = slot;
    return d;
}

static void fail_inflight(ServeState *S, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint64_t t : S->inflight) {
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) continue;
        it->second.state = 3;
        it->second.status = status;
    }
    S->inflight.clear();
}

static void serve_loop(ServeState *S) {
    fold_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    std::vector<uint64_t> admitted;
    int slice = 8;
    for (;;) {
        admitted.clear();
        std::vector<Request *> active;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->inflight.empty() && S->queued.empty())
                S->cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return S->stop || !S->queued.empty(); });
            if (S->stop) return;
            // admission: FIFO while the arena has room and the in-flight limit allows
            while (!S->queued.empty() && (int)S->inflight.size() < S->max_inflight) {
                Request &r = S->reqs[S->queued.front()];
                size_t off;
                if (!S->arena.alloc(r.bytes, &off)) break;
                r.block = off;
                r.state = 1;
                S->inflight.push_back(r.ticket);
                admitted.push_back(r.ticket);
                S->queued.pop_front();
            }
            for (uint64_t t : S->inflight) active.push_back(&S->reqs[t]);
        }
        if (active.empty()) continue;
        // new requests: zeroed control/flag region and padded codes
        cudaError_t e = cudaSuccess;
        for (uint64_t t : admitted) {
            Request *r;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                r = &S->reqs[t];
            }
            uint8_t *base = S->arena_base + r->block;
            if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, r->pl.zero_bytes, S->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(base + r->pl.off_codes, r->codes.data(), r->codes.size(), cudaMemcpyHostToDevice, S->st);
            // the host copy of the codes must stay alive until this copy ran: synchronised below
        }
        // one slice: kSlice steps of every active request, interleaved step by step
        std::vector<SeqDesc> sds(active.size());
        std::vector<int4> tasks;
        for (size_t k = 0; k < active.size(); ++k) sds[k] = arena_desc(*active[k], (int)k);
        for (int off = 0; off < slice; ++off) {
            for (size_t k = 0; k < active.size(); ++k) {
                const Request &r = *active[k];
                const int step = r.cursor + off;
                if (step >= r.NT) continue;
                for (int q = r.step_begin[step]; q < r.step_begin[step + 1]; ++q) {
                    int4 tk = r.tasks[q];
                    tk.x = (int)k;
                    tasks.push_back(tk);
                }
            }
        }
        const size_t cnt = active.size();
        const size_t o_res = 256, o_sd = al256(o_res + 4 * cnt), o_tasks = al256(o_sd + sizeof(SeqDesc) * cnt);
        const size_t o_out = al256(o_tasks + sizeof(int4) * tasks.size());
        const size_t total = al256(o_out + 4 * cnt);
        if (ensure_buf(S->d_launch, total) || ensure_host(S->h_launch, total)) {
            fail_inflight(S, FOLD_ENOMEM);
            continue;
        }
        uint8_t *h = reinterpret_cast<uint8_t *>(S->h_launch.ptr);
        uint8_t *d = reinterpret_cast<uint8_t *>(S->d_launch.ptr);
        memcpy(h + o_sd, sds.data(), sizeof(SeqDesc) * cnt);
        if (!tasks.empty()) memcpy(h + o_tasks, tasks.data(), sizeof(int4) * tasks.size());
        if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, o_sd, S->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_sd, h + o_sd, o_out - o_sd, cudaMemcpyHostToDevice, S->st);
        FoldParams p;
        memset(&p, 0, sizeof p);
        p.tasks = reinterpret_cast<const int4 *>(d + o_tasks);
        p.ntasks = (int)tasks.size();
        p.queue_head = reinterpret_cast<int *>(d);
        p.error = reinterpret_cast<int *>(d) + 1;
        p.queue_head_far = reinterpret_cast<int *>(d) + 2;
        p.nnear = 0;
        p.near_ctas = 0;
        p.seqs = reinterpret_cast<const SeqDesc *>(d + o_sd);
        p.codes = S->arena_base;
        p.drow = reinterpret_cast<int16_t *>(S->arena_base);
        p.dcol = reinterpret_cast<int16_t *>(S->arena_base);
        p.rf = reinterpret_cast<uint32_t *>(S->arena_base);
        p.cf = reinterpret_cast<uint32_t *>(S->arena_base);
        p.flags = reinterpret_cast<int *>(S->arena_base);
        p.cnt = reinterpret_cast<int *>(S->arena_base);
        p.pring = reinterpret_cast<int *>(S->arena_base);
        p.results = reinterpret_cast<int *>(d + o_res);
        p.rtab = ctx->d_rpacked;
        p.pair64 = ctx->pair64;
        p.timeout_ns = ctx->timeout_ms * 1000000LL;
        p.trace = nullptr;
        const auto t_launch = std::chrono::steady_clock::now();
        if (e == cudaSuccess && p.ntasks > 0) e = launch_fold(p, ctx->q, ctx->method, grid_for(ctx), S->st);
        if (e == cudaSuccess)
            e = launch_finalize(p.error, p.results, (int)cnt, reinterpret_cast<int32_t *>(d + o_out), S->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h + o_out, d + o_out, 4 * cnt, cudaMemcpyDeviceToHost, S->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
        S->launches += 3;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_launch).count();
        const int used = slice;
        slice = std::max(kSliceMin, std::min(kSliceMax, (int)(slice * kSliceTargetMs / std::max(ms, 0.05))));
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail_inflight(S, FOLD_ECUDA);
            continue;
        }
        const int32_t *hres = reinterpret_cast<const int32_t *>(h + o_out);
        std::lock_guard<std::mutex> lk(S->mu);
        std::vector<uint64_t> still;
        for (size_t k = 0; k < cnt; ++k) {
            Request &r = *active[k];
            if (hres[k] < 0) {   // a bounded device-side wait expired in this launch
                r.state = 3;
                r.status = -hres[k] == FOLD_ETIMEOUT ? FOLD_ETIMEOUT : FOLD_ECUDA;
                continue;
            }
            r.cursor += used;
            if (r.cursor >= r.NT) {
                r.state = 2;
                r.result = r.n >= 2 ? hres[k] : 0;
            } else {
                still.push_back(r.ticket);
            }
        }
        S->inflight.swap(still);
    }
}

}  // namespace fold

using namespace fold;

extern "C" {

int fold_serve_start(fold_ctx *ctx, int64_t budget_bytes, int32_t max_inflight) {
    if (!ctx || budget_bytes < (1 << 20) || max_inflight < 1) return FOLD_EINVAL;
    if (ctx->serve) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    ServeState *S = new ServeState();
    S->ctx = ctx;
    S->budget = (size_t)budget_bytes;
    S->max_inflight = max_inflight;
    if (cudaMalloc(&S->arena_base, S->budget) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return FOLD_ENOMEM;
    }
    S->arena.init(S->budget);
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->poll_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(S->arena_base);
        delete S;
        return FOLD_ECUDA;
    }
    ctx->serve = S;
    S->th = std::thread(serve_loop, S);
    return FOLD_OK;
}

int fold_serve_submit(fold_ctx *ctx, const char *seq, int32_t n, uint64_t *ticket) {
    if (!ctx || !ticket || n < 0 || n > FOLD_MAX_N || (n > 0 && !seq)) return FOLD_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return FOLD_EINVAL;
    Request r;
    r.n = n;
    r.pl = make_plan(&n, 1, ctx->q, ctx->method);
    r.NT = r.pl.NTs[0];
    r.bytes = r.pl.bytes;
    if (r.bytes > S->budget) return FOLD_EAGAIN;
    const int Np = r.pl.sd[0].Np;
    r.codes.assign((size_t)std::max(Np, 1), (uint8_t)kPadCode);
    if (!encode_seq(seq, n, r.codes.data())) return FOLD_EINVAL;
    if (n > 0) {
        int kc = ctx->kc_override > 0 ? ctx->kc_override : kc_auto(r.NT);
        build_schedule_steps(r.NT, kc, strip_of(ctx->q, ctx->method), r.tasks, r.step_begin);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->reqs.size() >= kMaxQueued) return FOLD_EAGAIN;
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    if (n == 0) {
        r.state = 2;
        r.result = 0;
        S->reqs.emplace(r.ticket, std::move(r));
        return FOLD_OK;
    }
    uint64_t t = r.ticket;
    S->reqs.emplace(t, std::move(r));
    S->queued.push_back(t);
    S->cv.notify_one();
    return FOLD_OK;
}

int fold_serve_poll(fold_ctx *ctx, uint64_t ticket, int32_t *max_pairs, int16_t *D_out) {
    if (!ctx || !max_pairs) return FOLD_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return FOLD_EINVAL;
    Request r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return FOLD_EINVAL;
        if (it->second.state == 0 || it->second.state == 1) return FOLD_ENOTREADY;
        r = std::move(it->second);
        S->reqs.erase(it);
    }
    int status = r.state == 2 ? FOLD_OK : r.status;
    if (status == FOLD_OK) *max_pairs = r.result;
    if (status == FOLD_OK && D_out && r.n > 0) {
        cudaSetDevice(ctx->device);
        int16_t *dd = nullptr;
        size_t bytes = (size_t)r.n * r.n * 2;
        cudaError_t e = cudaMalloc(&dd, bytes);
        if (e == cudaSuccess)
            e = launch_extract(reinterpret_cast<int16_t *>(S->arena_base + r.block + r.pl.off_drow), r.pl.sd[0].Np, r.n, dd,
                               S->poll_st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(D_out, dd, bytes, cudaMemcpyDeviceToHost, S->poll_st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->poll_st);
        if (dd) cudaFree(dd);
        if (e != cudaSuccess) status = status_from_cuda(e);
    }
    if (r.bytes && r.n > 0 && r.state != 0) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->arena.release(r.block, r.bytes);
        S->cv.notify_one();
    }
    return status;
}

int fold_serve_stop(fold_ctx *ctx) {
    if (!ctx) return FOLD_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return FOLD_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(S->st);
    cudaStreamSynchronize(S->poll_st);
    ctx->launches += S->launches;
    if (S->d_launch.ptr) cudaFree(S->d_launch.ptr);
    if (S->h_launch.ptr) cudaFreeHost(S->h_launch.ptr);
    cudaFree(S->arena_base);
    cudaStreamDestroy(S->st);
    cudaStreamDestroy(S->poll_st);
    delete S;
    ctx->serve = nullptr;
    return FOLD_OK;
}

}  // extern "C"
