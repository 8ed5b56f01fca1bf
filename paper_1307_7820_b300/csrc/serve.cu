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
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
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
constexpr int kSoloMaxN = 8192;      // a lone request up to this length folds in one launch (~3.5 ms)
constexpr size_t kMaxQueued = 1 << 20;
constexpr size_t kLaunchBytes0 = size_t(16) << 20;   // initial launch-list buffers (host and device)

struct Request {
    uint64_t ticket = 0;
    int n = 0;
    int NT = 0;
    std::vector<uint8_t> codes;      // padded to Np with the padding code
    Plan pl;
    size_t block = 0;                // arena byte offset
    size_t bytes = 0;
    std::shared_ptr<const SeqTemplate> sched;   // task list of a fold of this size, by step (shared)
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
    std::deque<uint64_t> done_q;     // finished tickets not yet reported by fold_serve_wait_any
    std::condition_variable done_cv;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    // launch buffers
    DevBuf d_launch;                 // control | results | SeqDesc | tasks
    HostBuf h_launch;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    unsigned long long launches = 0;
    fold_serve_stats stats{};        // guarded by mu
};

static size_t al256(size_t v) { return (v + 255) / 256 * 256; }
// capacity to ask for when `want` bytes are needed: at least double the current one, so that
// growing launch lists reallocate (and synchronise) only a few times
static size_t grown(size_t have, size_t want) { return want <= have ? have : std::max(want, 2 * have); }

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

// a request is done or failed (S->mu held): report it to fold_serve_wait_any
static void mark_done(ServeState *S, uint64_t ticket) {
    S->done_q.push_back(ticket);
    S->done_cv.notify_all();
}

static void fail_inflight(ServeState *S, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint64_t t : S->inflight) {
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) continue;
        it->second.state = 3;
        it->second.status = status;
        S->stats.finished++;
        mark_done(S, t);
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
        const auto t_prep = std::chrono::steady_clock::now();
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
        // a request alone in the system (just admitted, nothing else in flight or waiting) folds in
        // one launch with the single-fold work split (column mode where it applies), as
        // fold_score_dev would, instead of slice by slice in the one-queue layout; up to
        // kSoloMaxN, so that a request arriving meanwhile waits at most about that fold's time
        bool solo = false;
        if (e == cudaSuccess && active.size() == 1 && admitted.size() == 1 && active[0]->cursor == 0 &&
            active[0]->n >= 2 && active[0]->n <= kSoloMaxN) {
            std::lock_guard<std::mutex> lk(S->mu);
            solo = S->queued.empty();
        }
        if (solo) {
            Request &r = *active[0];
            const SeqTemplate &sc = *r.sched;
            const FoldOpts o;   // automatic work split, whatever the caller's options
            const SplitPlan sp = plan_split(ctx, o, r.NT, grid_for(ctx), true);
            const size_t nt = sc.tasks.size();
            // launch buffers: SeqDesc | result | tasks; with tile-only CTAs the list is split into
            // [tile tasks | chunks], each in the template's order (its tiles are by diagonal, as
            // column mode reads them): both parts are whole ranges of every step
            const size_t o_res = 256, o_tasks = 512, need = al256(o_tasks + sizeof(int4) * nt);
            if (ensure_buf(S->d_launch, grown(S->d_launch.bytes, need)) == FOLD_OK &&
                ensure_host(S->h_launch, grown(S->h_launch.bytes, need)) == FOLD_OK) {
                uint8_t *h = reinterpret_cast<uint8_t *>(S->h_launch.ptr);
                uint8_t *d = reinterpret_cast<uint8_t *>(S->d_launch.ptr);
                memcpy(h, &r.pl.sd[0], sizeof(SeqDesc));
                int4 *dst = reinterpret_cast<int4 *>(h + o_tasks);
                int nnear = 0;
                if (sp.near_ctas > 0) {
                    for (int t = 0; t < r.NT; ++t) {
                        const int a = sc.near_begin[t], b = sc.chunk_begin[t];
                        memcpy(dst, sc.tasks.data() + a, sizeof(int4) * (size_t)(b - a));
                        dst += b - a;
                        nnear += b - a;
                    }
                    for (int t = 0; t < r.NT; ++t) {
                        const int a = sc.chunk_begin[t], b = sc.near_begin[t + 1];
                        memcpy(dst, sc.tasks.data() + a, sizeof(int4) * (size_t)(b - a));
                        dst += b - a;
                    }
                } else {
                    memcpy(dst, sc.tasks.data(), sizeof(int4) * nt);
                }
                if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, sizeof(SeqDesc), cudaMemcpyHostToDevice, S->st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(d + o_tasks, h + o_tasks, sizeof(int4) * nt, cudaMemcpyHostToDevice, S->st);
                FoldParams p = make_params(ctx, r.pl, S->arena_base + r.block, reinterpret_cast<const int4 *>(d + o_tasks),
                                           (int)nt, reinterpret_cast<const SeqDesc *>(d));
                if (sp.near_ctas > 0) {
                    p.col_mode = sp.col_mode;
                    p.cols_per_cta = sp.cpc;
                    p.col_helpers = sp.helpers;
                    p.nnear = nnear;
                    p.near_ctas = sp.near_ctas;
                }
                int32_t *d_out = reinterpret_cast<int32_t *>(d + o_res);
                int32_t *h_out = reinterpret_cast<int32_t *>(h + o_res);
                const auto t_launch = std::chrono::steady_clock::now();
                if (e == cudaSuccess) e = cudaEventRecord(S->ev0, S->st);
                if (e == cudaSuccess) e = launch_fold(p, ctx->q, ctx->method, grid_for(ctx), S->st);
                if (e == cudaSuccess) e = launch_finalize(p.error, p.results, 1, d_out, S->st);
                if (e == cudaSuccess) e = cudaEventRecord(S->ev1, S->st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, sizeof(int32_t), cudaMemcpyDeviceToHost, S->st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
                S->launches += 2;
                const auto t_done = std::chrono::steady_clock::now();
                float gpu_ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&gpu_ms, S->ev0, S->ev1);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    fail_inflight(S, FOLD_ECUDA);
                    continue;
                }
                std::lock_guard<std::mutex> lk(S->mu);
                S->stats.slices++;
                S->stats.solo++;
                S->stats.tasks += (uint64_t)nt;
                S->stats.admitted += 1;
                S->stats.gpu_ms += gpu_ms;
                S->stats.slice_ms += std::chrono::duration<double, std::milli>(t_done - t_prep).count();
                S->stats.prep_ms += std::chrono::duration<double, std::milli>(t_launch - t_prep).count();
                S->stats.finished++;
                if (h_out[0] < 0) {   // a bounded device-side wait expired
                    r.state = 3;
                    r.status = -h_out[0] == FOLD_ETIMEOUT ? FOLD_ETIMEOUT : FOLD_ECUDA;
                } else {
                    r.state = 2;
                    r.result = h_out[0];
                }
                r.cursor = r.NT;
                mark_done(S, r.ticket);
                S->inflight.clear();
                continue;
            }
            // no room for the launch buffers: slices as for any request
        }
        // one slice: `slice` steps of every active request, interleaved step by step, gathered
        // straight into the pinned staging buffer (whole steps are contiguous in a template)
        const size_t cnt = active.size();
        size_t ntasks = 0;
        for (const Request *r : active) {
            const int lo = std::min(r->cursor, r->NT), hi = std::min(r->cursor + slice, r->NT);
            ntasks += (size_t)(r->sched->near_begin[hi] - r->sched->near_begin[lo]);
        }
        const size_t o_res = 256, o_sd = al256(o_res + 4 * cnt), o_tasks = al256(o_sd + sizeof(SeqDesc) * cnt);
        const size_t o_out = al256(o_tasks + sizeof(int4) * ntasks);
        const size_t total = al256(o_out + 4 * cnt);
        if (ensure_buf(S->d_launch, grown(S->d_launch.bytes, total)) ||
            ensure_host(S->h_launch, grown(S->h_launch.bytes, total))) {
            fail_inflight(S, FOLD_ENOMEM);
            continue;
        }
        uint8_t *h = reinterpret_cast<uint8_t *>(S->h_launch.ptr);
        uint8_t *d = reinterpret_cast<uint8_t *>(S->d_launch.ptr);
        SeqDesc *hsd = reinterpret_cast<SeqDesc *>(h + o_sd);
        for (size_t k = 0; k < cnt; ++k) hsd[k] = arena_desc(*active[k], (int)k);
        int4 *dst = reinterpret_cast<int4 *>(h + o_tasks);
        for (int off = 0; off < slice; ++off) {
            for (size_t k = 0; k < cnt; ++k) {
                const Request &r = *active[k];
                const int step = r.cursor + off;
                if (step >= r.NT) continue;
                const SeqTemplate &sc = *r.sched;
                const int a = sc.near_begin[step], b = sc.near_begin[step + 1];
                if (k == 0) {   // templates carry sequence index 0
                    memcpy(dst, sc.tasks.data() + a, sizeof(int4) * (size_t)(b - a));
                } else {
                    for (int q = a; q < b; ++q) {
                        int4 tk = sc.tasks[q];
                        tk.x = (int)k;
                        dst[q - a] = tk;
                    }
                }
                dst += b - a;
            }
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, o_sd, S->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_sd, h + o_sd, o_out - o_sd, cudaMemcpyHostToDevice, S->st);
        FoldParams p;
        memset(&p, 0, sizeof p);
        p.tasks = reinterpret_cast<const int4 *>(d + o_tasks);
        p.ntasks = (int)ntasks;
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
        p.memo = (ctx->r_memo && ctx->method == kTwoVector) ? 1 : 0;
        p.timeout_ns = ctx->timeout_ms * 1000000LL;
        p.trace = nullptr;
        const auto t_launch = std::chrono::steady_clock::now();
        if (e == cudaSuccess) e = cudaEventRecord(S->ev0, S->st);
        if (e == cudaSuccess && p.ntasks > 0) e = launch_fold(p, ctx->q, ctx->method, grid_for(ctx), S->st);
        if (e == cudaSuccess)
            e = launch_finalize(p.error, p.results, (int)cnt, reinterpret_cast<int32_t *>(d + o_out), S->st);
        if (e == cudaSuccess) e = cudaEventRecord(S->ev1, S->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h + o_out, d + o_out, 4 * cnt, cudaMemcpyDeviceToHost, S->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
        S->launches += 3;
        const auto t_done = std::chrono::steady_clock::now();
        const double ms = std::chrono::duration<double, std::milli>(t_done - t_launch).count();
        float gpu_ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&gpu_ms, S->ev0, S->ev1);
        const int used = slice;
        slice = std::max(kSliceMin, std::min(kSliceMax, (int)(slice * kSliceTargetMs / std::max(ms, 0.05))));
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail_inflight(S, FOLD_ECUDA);
            continue;
        }
        const int32_t *hres = reinterpret_cast<const int32_t *>(h + o_out);
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.slices++;
        S->stats.tasks += (uint64_t)p.ntasks;
        S->stats.admitted += admitted.size();
        S->stats.gpu_ms += gpu_ms;
        S->stats.slice_ms += std::chrono::duration<double, std::milli>(t_done - t_prep).count();
        S->stats.prep_ms += std::chrono::duration<double, std::milli>(t_launch - t_prep).count();
        std::vector<uint64_t> still;
        for (size_t k = 0; k < cnt; ++k) {
            Request &r = *active[k];
            if (hres[k] < 0) {   // a bounded device-side wait expired in this launch
                S->stats.finished++;
                r.state = 3;
                r.status = -hres[k] == FOLD_ETIMEOUT ? FOLD_ETIMEOUT : FOLD_ECUDA;
                mark_done(S, r.ticket);
                continue;
            }
            r.cursor += used;
            if (r.cursor >= r.NT) {
                r.state = 2;
                r.result = r.n >= 2 ? hres[k] : 0;
                S->stats.finished++;
                mark_done(S, r.ticket);
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
    if (ctx->serve || ctx->method >= kSliding) return FOLD_EINVAL;
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
        cudaStreamCreateWithFlags(&S->poll_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&S->ev0) != cudaSuccess || cudaEventCreate(&S->ev1) != cudaSuccess) {
        cudaGetLastError();
        if (S->ev0) cudaEventDestroy(S->ev0);
        if (S->st) cudaStreamDestroy(S->st);
        if (S->poll_st) cudaStreamDestroy(S->poll_st);
        cudaFree(S->arena_base);
        delete S;
        return FOLD_ECUDA;
    }
    // launch lists of up to about a million tasks without reallocating (a reallocation synchronises)
    if (ensure_buf(S->d_launch, kLaunchBytes0) || ensure_host(S->h_launch, kLaunchBytes0)) {
        if (S->d_launch.ptr) cudaFree(S->d_launch.ptr);
        cudaEventDestroy(S->ev0);
        cudaEventDestroy(S->ev1);
        cudaStreamDestroy(S->st);
        cudaStreamDestroy(S->poll_st);
        cudaFree(S->arena_base);
        delete S;
        return FOLD_ENOMEM;
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
        const int kc = ctx->kc_override > 0 ? ctx->kc_override : kc_auto(r.NT);
        r.sched = seq_template(r.NT, kc, strip_of(ctx->q, ctx->method), true);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->reqs.size() >= kMaxQueued) return FOLD_EAGAIN;
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    if (n == 0) {
        r.state = 2;
        r.result = 0;
        const uint64_t t0 = r.ticket;
        S->reqs.emplace(t0, std::move(r));
        mark_done(S, t0);
        return FOLD_OK;
    }
    uint64_t t = r.ticket;
    S->reqs.emplace(t, std::move(r));
    S->queued.push_back(t);
    S->cv.notify_one();
    return FOLD_OK;
}

int fold_serve_wait_any(fold_ctx *ctx, int32_t timeout_ms, uint64_t *ticket) {
    if (!ctx || !ticket || timeout_ms < 0) return FOLD_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return FOLD_EINVAL;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (!S->done_q.empty()) {
            const uint64_t t = S->done_q.front();
            S->done_q.pop_front();
            if (S->reqs.count(t)) {   // tickets already polled are skipped
                *ticket = t;
                return FOLD_OK;
            }
        }
        if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && S->done_q.empty())
            return FOLD_ENOTREADY;
    }
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

int fold_serve_warm(fold_ctx *ctx, int32_t max_n) {
    if (!ctx || max_n < 0 || max_n > FOLD_MAX_N || ctx->method >= kSliding) return FOLD_EINVAL;
    if (max_n == 0) return FOLD_OK;
    int n = max_n;
    const int NTmax = make_plan(&n, 1, ctx->q, ctx->method).NTs[0];
    const int strip = strip_of(ctx->q, ctx->method), kco = ctx->kc_override;
    // largest first, so the threads finish together
    std::atomic<int> next(NTmax);
    auto work = [&] {
        for (int NT; (NT = next.fetch_sub(1)) >= 1;) seq_template(NT, kco > 0 ? kco : kc_auto(NT), strip, true);
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const int nth = (int)std::max(1u, std::min(hw, 16u));
    std::vector<std::thread> th;
    for (int k = 1; k < nth; ++k) th.emplace_back(work);
    work();
    for (auto &x : th) x.join();
    return FOLD_OK;
}

int fold_serve_stats_get(fold_ctx *ctx, fold_serve_stats *out) {
    if (!ctx || !out || !ctx->serve) return FOLD_EINVAL;
    ServeState *S = ctx->serve;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->queued = (int32_t)S->queued.size();
    out->inflight = (int32_t)S->inflight.size();
    return FOLD_OK;
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
    cudaEventDestroy(S->ev0);
    cudaEventDestroy(S->ev1);
    delete S;
    ctx->serve = nullptr;
    return FOLD_OK;
}

}  // extern "C"
