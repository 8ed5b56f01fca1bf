// serve.cu -- continuous-batching serving loop of libfold_b300.
//
// A host scheduler thread owns one device arena of `budget_bytes`.  Submitted
// requests wait in a FIFO until their workspace (D copies, difference
// vectors, tile flags: the single-sequence plan) fits the arena and fewer
// than `max_inflight` requests are in flight; a long request (at least
// FOLD_OPT_SERVE_LONG_TILES tiles per side) also waits while
// FOLD_OPT_SERVE_LONG_CAP long ones are in flight, and shorter requests behind
// it are admitted past it.  A request arriving to an idle
// server (up to kSoloMaxN bases) folds alone in one launch with the single
// fold's work split.  Otherwise the in-flight requests are folded by one
// persistent launch fed while it runs (the serving ring): the thread
// publishes, round after round, the next tile diagonal of every in-flight
// request's task list (the ordered list a single fold uses) into a device
// ring by copies, and advances the ring's tail; the launch's warps take tasks
// in ring order, each waiting (bounded) only on tasks of its own request
// published before it.  A request admitted meanwhile joins the next round, so
// no request waits for a launch boundary.  Answers come back through
// host-mapped memory; when nothing is in flight the thread stops the launch.
// With the ring switched off (FOLD_OPT_SERVE_RING = 0) the in-flight requests
// are folded in repeated launches instead, each advancing every request by a
// slice of tile diagonals.  All in-flight DP state stays in the arena.  A
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
constexpr int kRingCap = 1 << 22;    // serving ring: tasks (64 MiB)
constexpr long long kRingAhead = 8192;   // tasks published ahead of the claims the launch reported
constexpr int kResultPending = INT32_MIN;
constexpr size_t kSoloListBytes = size_t(256) << 20;   // device copies of lone requests' task lists
constexpr size_t kAdmitScan = 256;   // queued requests looked at per admission pass

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
    int slot = -1;                   // serving ring: index of its descriptor and answer
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
    int long_tiles = 0;              // requests of at least this many tiles per side are long (0: none)
    int long_cap = 0;                // ... and at most this many of them are in flight at once
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
    int near_ctas = 0;               // slices: tile-only CTAs (0: one shared queue)
    std::vector<int4> split_tmp;     // chunk tasks while a slice's list is split
    // serving ring
    bool use_ring = true;
    bool ring_on = false;            // a ring launch is running
    int ring_slots = 0;              // descriptors / answers (max_inflight)
    DevBuf d_ring;                   // control words | SeqDesc[ring_slots] | tasks[kRingCap]
    int *h_map = nullptr;            // host-mapped: answers[ring_slots] | reported claim index
    int *d_map = nullptr;            // its device address
    HostBuf h_stage;                 // pinned: a round's tasks, descriptors, codes, tail values
    HostBuf h_zero;                  // pinned zeros (a request's control region is cleared by a copy)
    cudaStream_t cst = nullptr;      // copies into the running launch
    cudaEvent_t ring_ev0 = nullptr, ring_ev1 = nullptr;
    long long ring_tail = 0;         // tasks published
    std::vector<int> free_slots;
    std::chrono::steady_clock::time_point ring_t0;
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


// ---------------------------------------------------------------- serving ring
// Device layout of d_ring: control words (queue head, error, tail, stop) | SeqDesc per slot | tasks.
static constexpr size_t kRingCtrl = 256;
static size_t ring_o_sd() { return kRingCtrl; }
static size_t ring_o_tasks(const ServeState *S) { return al256(kRingCtrl + sizeof(SeqDesc) * (size_t)S->ring_slots); }
static constexpr size_t kStageBytes = size_t(32) << 20;   // pinned staging per batch of copies
static constexpr size_t kZeroBytes = size_t(16) << 20;    // pinned zeros, copied as often as needed

// Resources for the ring, made when serving starts (nothing here may allocate or free while a ring
// launch runs: those calls can wait for the device, which waits for this thread).
static int ring_setup(ServeState *S) {
    S->ring_slots = S->max_inflight;
    const size_t bytes = ring_o_tasks(S) + sizeof(int4) * (size_t)kRingCap;
    if (ensure_buf(S->d_ring, bytes)) return FOLD_ENOMEM;
    if (cudaHostAlloc(reinterpret_cast<void **>(&S->h_map), sizeof(int) * ((size_t)S->ring_slots + 64),
                      cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return FOLD_ENOMEM;
    }
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&S->d_map), S->h_map, 0) != cudaSuccess) {
        cudaGetLastError();
        return FOLD_ECUDA;
    }
    if (ensure_host(S->h_stage, kStageBytes) || ensure_host(S->h_zero, kZeroBytes)) return FOLD_ENOMEM;
    memset(S->h_zero.ptr, 0, kZeroBytes);
    if (cudaStreamCreateWithFlags(&S->cst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&S->ring_ev0) != cudaSuccess || cudaEventCreate(&S->ring_ev1) != cudaSuccess) {
        cudaGetLastError();
        return FOLD_ECUDA;
    }
    S->free_slots.clear();
    for (int k = S->ring_slots - 1; k >= 0; --k) S->free_slots.push_back(k);
    return FOLD_OK;
}

static void ring_teardown(ServeState *S) {
    if (S->cst) cudaStreamDestroy(S->cst);
    if (S->ring_ev0) cudaEventDestroy(S->ring_ev0);
    if (S->ring_ev1) cudaEventDestroy(S->ring_ev1);
    if (S->h_map) cudaFreeHost(S->h_map);
    if (S->h_stage.ptr) cudaFreeHost(S->h_stage.ptr);
    if (S->h_zero.ptr) cudaFreeHost(S->h_zero.ptr);
    if (S->d_ring.ptr) cudaFree(S->d_ring.ptr);
}

// One persistent launch over the ring, on S->st (its control words cleared first: no launch runs).
static cudaError_t ring_start(ServeState *S) {
    fold_ctx *ctx = S->ctx;
    uint8_t *base = reinterpret_cast<uint8_t *>(S->d_ring.ptr);
    int *ctrl = reinterpret_cast<int *>(base);
    // cleared before any copy of the copy stream can reach the control words (the tail)
    cudaError_t e = cudaMemsetAsync(ctrl, 0, kRingCtrl, S->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    reinterpret_cast<volatile int *>(S->h_map)[S->ring_slots] = 0;   // claim index reported so far
    FoldParams p;
    memset(&p, 0, sizeof p);
    p.tasks = reinterpret_cast<const int4 *>(base + ring_o_tasks(S));
    p.ntasks = 0;
    p.queue_head = ctrl;
    p.error = ctrl + 1;
    p.queue_head_far = ctrl + 4;
    p.seqs = reinterpret_cast<const SeqDesc *>(base + ring_o_sd());
    p.codes = S->arena_base;
    p.drow = reinterpret_cast<int16_t *>(S->arena_base);
    p.dcol = reinterpret_cast<int16_t *>(S->arena_base);
    p.rf = reinterpret_cast<uint32_t *>(S->arena_base);
    p.cf = reinterpret_cast<uint32_t *>(S->arena_base);
    p.flags = reinterpret_cast<int *>(S->arena_base);
    p.cnt = reinterpret_cast<int *>(S->arena_base);
    p.pring = reinterpret_cast<int *>(S->arena_base);
    p.results = S->d_map;
    p.rtab = ctx->d_rpacked;
    p.pair64 = ctx->pair64;
    p.memo = (ctx->r_memo && ctx->method == kTwoVector) ? 1 : 0;
    p.timeout_ns = ctx->timeout_ms * 1000000LL;
    p.ring_cap = kRingCap;
    p.ring_tail = ctrl + 2;
    p.ring_stop = ctrl + 3;
    p.ring_progress = S->d_map + S->ring_slots;
    if (e == cudaSuccess) e = cudaEventRecord(S->ring_ev0, S->st);
    if (e == cudaSuccess) e = launch_fold(p, ctx->q, ctx->method, grid_for(ctx), S->st);
    if (e == cudaSuccess) e = cudaEventRecord(S->ring_ev1, S->st);
    if (e == cudaSuccess) {
        S->ring_on = true;
        S->ring_tail = 0;
        S->launches += 1;
        S->ring_t0 = std::chrono::steady_clock::now();
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.slices++;
    }
    return e;
}

// The device copy of a lone request's task list (template sc of NT tiles per side; with split, as
// [tile tasks | chunk tasks], each in the template's order -- its tiles by diagonal, as column mode
// reads them -- both parts whole ranges of every step), from the context's cache or built now
// through `staging` on stream st.  *out receives the entry (dev null if it could not be made).
// Making room drops the least recently used lists, which only the serving thread may do (may_evict),
// and only while no launch is in flight: another thread could free a list between its lookup and its
// launch.
static cudaError_t solo_list(fold_ctx *ctx, int NT, const SeqTemplate &sc, bool split, HostBuf *staging,
                             cudaStream_t st, bool may_evict, SoloList *out) {
    *out = SoloList();
    const auto key = std::make_tuple(NT, ctx->kc_override > 0 ? ctx->kc_override : kc_auto(NT), split);
    std::lock_guard<std::mutex> lk(ctx->solo_mu);
    auto it = ctx->solo_lists.find(key);
    if (it != ctx->solo_lists.end()) {
        it->second.used = ++ctx->solo_clock;
        *out = it->second;
        return cudaSuccess;
    }
    const size_t nt = sc.tasks.size(), bytes = al256(sizeof(int4) * std::max<size_t>(nt, 1));
    if (!may_evict && ctx->solo_list_bytes + bytes > kSoloListBytes) return cudaSuccess;
    if (ensure_host(*staging, grown(staging->bytes, bytes)) != FOLD_OK) return cudaSuccess;
    while (!ctx->solo_lists.empty() && ctx->solo_list_bytes + bytes > kSoloListBytes) {
        auto victim = ctx->solo_lists.begin();
        for (auto v = ctx->solo_lists.begin(); v != ctx->solo_lists.end(); ++v)
            if (v->second.used < victim->second.used) victim = v;
        cudaFree(victim->second.dev);
        ctx->solo_list_bytes -= victim->second.bytes;
        ctx->solo_lists.erase(victim);
    }
    SoloList L;
    if (cudaMalloc(&L.dev, bytes) != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    int4 *dst = reinterpret_cast<int4 *>(staging->ptr);
    if (split) {
        for (int t = 0; t < NT; ++t) {
            const int a = sc.near_begin[t], b = sc.chunk_begin[t];
            memcpy(dst, sc.tasks.data() + a, sizeof(int4) * (size_t)(b - a));
            dst += b - a;
            L.nnear += b - a;
        }
        for (int t = 0; t < NT; ++t) {
            const int a = sc.chunk_begin[t], b = sc.near_begin[t + 1];
            memcpy(dst, sc.tasks.data() + a, sizeof(int4) * (size_t)(b - a));
            dst += b - a;
        }
    } else {
        memcpy(dst, sc.tasks.data(), sizeof(int4) * nt);
    }
    L.bytes = bytes;
    L.ntasks = (int)nt;
    cudaError_t e = cudaMemcpyAsync(L.dev, staging->ptr, sizeof(int4) * nt, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the staging is reused
    if (e != cudaSuccess) {
        cudaFree(L.dev);
        return e;
    }
    L.used = ++ctx->solo_clock;
    ctx->solo_lists.emplace(key, L);
    ctx->solo_list_bytes += bytes;
    *out = L;
    return cudaSuccess;
}

// Copies `bytes` from pinned staging (or zeros) to the device on the copy stream, in pieces the
// pinned buffers hold; the caller synchronises the copy stream before reusing the staging.
static cudaError_t ring_zero(ServeState *S, uint8_t *dst, size_t bytes) {
    cudaError_t e = cudaSuccess;
    for (size_t o = 0; o < bytes && e == cudaSuccess; o += kZeroBytes)
        e = cudaMemcpyAsync(dst + o, S->h_zero.ptr, std::min(kZeroBytes, bytes - o), cudaMemcpyHostToDevice, S->cst);
    return e;
}

// A newly admitted request on the ring: its slot, answer word, descriptor, cleared control region and
// codes (copies on the copy stream, all before any of its tasks is published).
static cudaError_t ring_admit(ServeState *S, Request &r, uint8_t *stage, size_t *used) {
    r.slot = S->free_slots.back();
    S->free_slots.pop_back();
    reinterpret_cast<volatile int *>(S->h_map)[r.slot] = kResultPending;
    uint8_t *base = S->arena_base + r.block;
    SeqDesc d = arena_desc(r, r.slot);
    const size_t need = al256(sizeof(SeqDesc)) + al256(r.codes.size());
    if (*used + need > kStageBytes) {   // staging full: let the copies queued so far finish
        cudaError_t e = cudaStreamSynchronize(S->cst);
        if (e != cudaSuccess) return e;
        *used = 0;
    }
    uint8_t *hs = stage + *used;
    memcpy(hs, &d, sizeof d);
    memcpy(hs + al256(sizeof(SeqDesc)), r.codes.data(), r.codes.size());
    *used += need;
    uint8_t *dsd = reinterpret_cast<uint8_t *>(S->d_ring.ptr) + ring_o_sd() + sizeof(SeqDesc) * (size_t)r.slot;
    cudaError_t e = cudaMemcpyAsync(dsd, hs, sizeof(SeqDesc), cudaMemcpyHostToDevice, S->cst);
    if (e == cudaSuccess) e = ring_zero(S, base, r.pl.zero_bytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + r.pl.off_codes, hs + al256(sizeof(SeqDesc)), r.codes.size(), cudaMemcpyHostToDevice, S->cst);
    return e;
}

// Publishes rounds (the next tile diagonal of every in-flight request, in admission order) while
// fewer than kRingAhead tasks are published beyond the claims the launch reported; returns the tasks
// published.
static long long ring_publish(ServeState *S, const std::vector<Request *> &active, uint8_t *stage, size_t used,
                              cudaError_t *err) {
    const long long claimed = reinterpret_cast<volatile int *>(S->h_map)[S->ring_slots];
    int4 *buf = reinterpret_cast<int4 *>(stage + al256(used));
    const size_t cap = (kStageBytes - al256(used) - 256) / sizeof(int4);
    size_t m = 0;
    // one diagonal of every request per round (a round's tasks are mostly ready to run when claimed:
    // more diagonals per round for long requests filled the queue with waiting chunks and collapsed the
    // throughput at 2000 req/s), the requests with the most diagonals left first, so the long ones,
    // whose chains set the tail latency, are claimed at the head of each round
    std::vector<Request *> order(active.begin(), active.end());
    std::stable_sort(order.begin(), order.end(),
                     [](const Request *x, const Request *y) { return x->NT - x->cursor > y->NT - y->cursor; });
    bool any = true;
    while (any && S->ring_tail + (long long)m - claimed < kRingAhead) {
        any = false;
        for (Request *r : order) {
            if (r->cursor >= r->NT) continue;
            const int steps = 1;
            const SeqTemplate &sc = *r->sched;
            const int a = sc.near_begin[r->cursor], b = sc.near_begin[r->cursor + steps];
            if (m + (size_t)(b - a) > cap) break;
            for (int q = a; q < b; ++q) {
                int4 tk = sc.tasks[q];
                tk.x = r->slot;
                buf[m++] = tk;
            }
            r->cursor += steps;
            any = true;
        }
    }
    if (m == 0) return 0;
    int4 *ring = reinterpret_cast<int4 *>(reinterpret_cast<uint8_t *>(S->d_ring.ptr) + ring_o_tasks(S));
    const size_t at = (size_t)(S->ring_tail % kRingCap);
    const size_t first = std::min(m, (size_t)kRingCap - at);
    cudaError_t e = cudaMemcpyAsync(ring + at, buf, sizeof(int4) * first, cudaMemcpyHostToDevice, S->cst);
    if (e == cudaSuccess && first < m)
        e = cudaMemcpyAsync(ring, buf + first, sizeof(int4) * (m - first), cudaMemcpyHostToDevice, S->cst);
    int *tail_src = reinterpret_cast<int *>(buf + m);
    *tail_src = (int)(S->ring_tail + (long long)m);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(reinterpret_cast<int *>(S->d_ring.ptr) + 2, tail_src, sizeof(int), cudaMemcpyHostToDevice, S->cst);
    *err = e;
    if (e == cudaSuccess) S->ring_tail += (long long)m;
    return (long long)m;
}

// Fails every in-flight request of the ring and frees their slots.
static void ring_fail(ServeState *S, int status) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (uint64_t t : S->inflight) {
            auto it = S->reqs.find(t);
            if (it != S->reqs.end() && it->second.slot >= 0) S->free_slots.push_back(it->second.slot);
        }
    }
    fail_inflight(S, status);
}

// Stops the ring launch (no more tasks) and waits for it; returns its error word.
static int ring_stop(ServeState *S) {
    int *stop_src = reinterpret_cast<int *>(S->h_stage.ptr);
    *stop_src = 1;
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<int *>(S->d_ring.ptr) + 3, stop_src, sizeof(int),
                                    cudaMemcpyHostToDevice, S->cst);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->cst);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, reinterpret_cast<int *>(S->d_ring.ptr) + 1, sizeof(int), cudaMemcpyDeviceToHost);
    S->ring_on = false;
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, S->ring_ev0, S->ring_ev1);
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.gpu_ms += ms;
    S->stats.slice_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - S->ring_t0).count();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return kErrTimeout;
    }
    return err;
}

// One pass of the ring loop over the in-flight requests: admit the new ones, publish rounds, collect
// answers; the launch starts when needed and stops when nothing is in flight.
static void ring_iteration(ServeState *S, const std::vector<uint64_t> &admitted, std::vector<Request *> &active) {
    cudaError_t e = cudaSuccess;
    uint8_t *stage = reinterpret_cast<uint8_t *>(S->h_stage.ptr) + 256;   // the first 256 bytes: the stop word
    size_t used = 0;
    const auto t_prep = std::chrono::steady_clock::now();
    for (uint64_t t : admitted) {
        Request *r;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r = &S->reqs[t];
        }
        if (e == cudaSuccess) e = ring_admit(S, *r, stage, &used);
    }
    if (e == cudaSuccess && !S->ring_on) e = ring_start(S);
    long long pub = 0;
    if (e == cudaSuccess) pub = ring_publish(S, active, stage, used, &e);
    if (e == cudaSuccess && (used || pub)) e = cudaStreamSynchronize(S->cst);   // the staging is free again
    const auto t_pub = std::chrono::steady_clock::now();
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (S->ring_on) ring_stop(S);
        ring_fail(S, FOLD_ECUDA);
        return;
    }
    // answers (host-mapped, written behind a system-scope fence by each request's last tile)
    const volatile int *ans = S->h_map;
    bool launch_ended = cudaEventQuery(S->ring_ev1) == cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.tasks += (uint64_t)pub;
        S->stats.admitted += admitted.size();
        S->stats.prep_ms += std::chrono::duration<double, std::milli>(t_pub - t_prep).count();
        std::vector<uint64_t> still;
        for (uint64_t t : S->inflight) {
            Request &r = S->reqs[t];
            const int v = ans[r.slot];
            if (v != kResultPending) {
                if (v < 0) {
                    r.state = 3;
                    r.status = FOLD_ECUDA;
                } else {
                    r.state = 2;
                    r.result = r.n >= 2 ? v : 0;
                }
                S->free_slots.push_back(r.slot);
                S->stats.finished++;
                mark_done(S, t);
            } else {
                still.push_back(t);
            }
        }
        S->inflight.swap(still);
        launch_ended = launch_ended && !S->inflight.empty();
    }
    if (launch_ended) {   // the launch left with requests unanswered: a bounded wait expired
        const int err = ring_stop(S);
        ring_fail(S, err == kErrTimeout ? FOLD_ETIMEOUT : FOLD_ECUDA);
        return;
    }
    bool idle;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        idle = S->inflight.empty() && S->queued.empty();
    }
    if (idle) {
        ring_stop(S);
        return;
    }
    if (!pub && admitted.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
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
            // admission: in arrival order while the arena has room and the in-flight limit allows.
            // Long requests (at least long_tiles tiles per side) beyond long_cap in flight wait, in
            // their order, and shorter ones behind them are admitted past them: in flight, requests
            // share the launch round by round, so every long one admitted slows the others.
            int nlong = 0;
            if (S->long_tiles > 0)
                for (uint64_t t : S->inflight) nlong += S->reqs[t].NT >= S->long_tiles ? 1 : 0;
            size_t qi = 0;
            while (qi < S->queued.size() && qi < kAdmitScan && (int)S->inflight.size() < S->max_inflight) {
                Request &r = S->reqs[S->queued[qi]];
                const bool is_long = S->long_tiles > 0 && r.NT >= S->long_tiles;
                if (is_long && nlong >= S->long_cap) {
                    ++qi;
                    continue;
                }
                size_t off;
                if (!S->arena.alloc(r.bytes, &off)) break;   // memory: no request passes another
                r.block = off;
                r.state = 1;
                S->inflight.push_back(r.ticket);
                admitted.push_back(r.ticket);
                S->queued.erase(S->queued.begin() + (std::ptrdiff_t)qi);
                nlong += is_long ? 1 : 0;
            }
            for (uint64_t t : S->inflight) active.push_back(&S->reqs[t]);
        }
        if (active.empty()) {
            if (S->ring_on) ring_stop(S);   // nothing to publish: the launch must not wait for tasks
            continue;
        }
        // a request alone in the system (just admitted, nothing else in flight or waiting) folds in
        // one launch with the single-fold work split (column mode where it applies), as
        // fold_score_dev would, instead of on the ring or slice by slice in the one-queue layout; up
        // to kSoloMaxN, so that a request arriving meanwhile waits at most about that fold's time
        bool solo = false;
        if (!S->ring_on && active.size() == 1 && admitted.size() == 1 && active[0]->cursor == 0 &&
            active[0]->n >= 2 && active[0]->n <= kSoloMaxN) {
            std::lock_guard<std::mutex> lk(S->mu);
            solo = S->queued.empty();
        }
        if (S->use_ring && !solo) {
            ring_iteration(S, admitted, active);
            continue;
        }
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
        if (solo && e == cudaSuccess) {
            Request &r = *active[0];
            const SeqTemplate &sc = *r.sched;
            const FoldOpts o;   // automatic work split, whatever the caller's options
            const SplitPlan sp = plan_split(ctx, o, r.NT, grid_for(ctx), true);
            const size_t nt = sc.tasks.size();
            // the list on the device, built at first use of the size (or by fold_serve_warm)
            SoloList L;
            e = solo_list(ctx, r.NT, sc, sp.near_ctas > 0, &S->h_launch, S->st, true, &L);
            // launch buffers: SeqDesc | result
            const size_t o_res = 256, need = 512;
            if (e == cudaSuccess && L.dev && ensure_buf(S->d_launch, grown(S->d_launch.bytes, need)) == FOLD_OK &&
                ensure_host(S->h_launch, grown(S->h_launch.bytes, need)) == FOLD_OK) {
                const int nnear = L.nnear;
                uint8_t *h = reinterpret_cast<uint8_t *>(S->h_launch.ptr);
                uint8_t *d = reinterpret_cast<uint8_t *>(S->d_launch.ptr);
                memcpy(h, &r.pl.sd[0], sizeof(SeqDesc));
                if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, sizeof(SeqDesc), cudaMemcpyHostToDevice, S->st);
                FoldParams p = make_params(ctx, r.pl, S->arena_base + r.block, reinterpret_cast<const int4 *>(L.dev),
                                           (int)nt, reinterpret_cast<const SeqDesc *>(d));
                if (sp.near_ctas > 0) {
                    p.col_mode = sp.col_mode;
                    p.cols_per_cta = sp.cpc;
                    p.col_helpers = sp.helpers;
                    p.col_join = sp.join;
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
        // with tile-only CTAs (FOLD_OPT_NEAR_CTAS > 0 when serving started) the slice's list becomes
        // [tile tasks | chunk tasks], each part in list order; both queues are taken in order and a
        // task waits only on tasks before it in the list, so progress is kept as for a single fold's
        // split layout.  Measured slower than one shared queue at 1000-2000 req/s (p99 17 and 41 ms
        // against 10 and 14 ms: the chunk CTAs fall behind), so not the default
        int nnear = 0;
        const int grid = grid_for(ctx);
        const int near_ctas = S->near_ctas;
        const bool split = near_ctas > 0 && near_ctas < grid && ntasks > 0;
        if (split) {
            int4 *all = reinterpret_cast<int4 *>(h + o_tasks);
            S->split_tmp.resize(ntasks);
            int4 *far = S->split_tmp.data();
            size_t nf = 0;
            for (size_t q = 0; q < ntasks; ++q) {
                if (task_type(all[q].y) == kTaskNear) all[nnear++] = all[q];
                else far[nf++] = all[q];
            }
            memcpy(all + nnear, far, sizeof(int4) * nf);
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
        p.nnear = split ? nnear : 0;
        p.near_ctas = split ? near_ctas : 0;
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
    S->long_tiles = ctx->serve_long_cap > 0 ? ctx->serve_long_tiles : 0;
    S->long_cap = ctx->serve_long_cap;
    S->near_ctas = ctx->near_ctas_opt > 0 ? ctx->near_ctas_opt : 0;
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
    S->use_ring = ctx->serve_ring != 0;
    if (S->use_ring) {
        const int rc = ring_setup(S);
        if (rc) {
            ring_teardown(S);
            if (S->d_launch.ptr) cudaFree(S->d_launch.ptr);
            if (S->h_launch.ptr) cudaFreeHost(S->h_launch.ptr);
            cudaEventDestroy(S->ev0);
            cudaEventDestroy(S->ev1);
            cudaStreamDestroy(S->st);
            cudaStreamDestroy(S->poll_st);
            cudaFree(S->arena_base);
            delete S;
            return rc;
        }
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
        // rows of the padded row-major table straight to the caller's buffer by the copy engine (no
        // kernel and no allocation: a ring launch may hold every SM), then the lower triangle, which
        // the fold never writes, set to zero
        cudaSetDevice(ctx->device);
        const size_t n = (size_t)r.n;
        cudaError_t e = cudaMemcpy2DAsync(D_out, n * 2, S->arena_base + r.block + r.pl.off_drow,
                                          (size_t)r.pl.sd[0].Np * 2, n * 2, n, cudaMemcpyDeviceToHost, S->poll_st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->poll_st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = status_from_cuda(e);
        } else {
            for (size_t i = 1; i < n; ++i) memset(D_out + i * n, 0, i * 2);
        }
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
    // the device copies of the lists a lone request launches with (lengths up to kSoloMaxN), in the
    // layout of the automatic work split, through a stream that waits on no other
    int ns = std::min(max_n, kSoloMaxN);
    const int NTsolo = make_plan(&ns, 1, ctx->q, ctx->method).NTs[0];
    cudaSetDevice(ctx->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return FOLD_ECUDA;
    HostBuf staging;
    cudaError_t e = cudaSuccess;
    for (int NT = 2; NT <= NTsolo && e == cudaSuccess; ++NT) {
        const SplitPlan sp = plan_split(ctx, FoldOpts(), NT, grid_for(ctx), true);
        SoloList L;
        e = solo_list(ctx, NT, *seq_template(NT, kco > 0 ? kco : kc_auto(NT), strip, true), sp.near_ctas > 0, &staging,
                      st, false, &L);
    }
    cudaStreamDestroy(st);
    if (staging.ptr) cudaFreeHost(staging.ptr);
    return e == cudaSuccess ? FOLD_OK : FOLD_ECUDA;
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
    if (S->ring_on) ring_stop(S);
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
    ring_teardown(S);
    delete S;
    ctx->serve = nullptr;
    return FOLD_OK;
}

}  // extern "C"
