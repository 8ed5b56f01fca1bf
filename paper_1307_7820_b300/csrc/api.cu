// api.cu -- C-ABI of libfold_b300 (declared in include/fold.h): context,
// workspace planning, single and batched folds.  Serving lives in serve.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/fold.h"
#include "api_internal.h"
#include "fold_common.h"
#include "kernels.h"
#include "schedule.h"
#include "fg.h"
#include "sliding.h"

using namespace fold;

namespace fold {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int kc_auto(int NT) { return std::min(64, std::max(4, NT / 18)); }

// Layout of `count` sequences inside one workspace.  Sections (256-byte
// aligned): control | results | flags | counters | P ring | codes | Drow |
// Dcol | row features | column features.  The first five are zeroed before
// every launch.
Plan make_plan(const int32_t *lens, int count, int q, int method) {
    Plan pl;
    pl.q = q;
    pl.method = method;
    pl.T = tile_of(q, method);
    pl.count = count;
    const int T = pl.T;
    size_t o_code = 0, o_drow = 0, o_dcol = 0, o_rf = 0, o_cf = 0, o_flag = 0, o_cnt = 0, o_p = 0;
    pl.sd.resize(count);
    pl.NTs.resize(count);
    for (int k = 0; k < count; ++k) {
        SeqDesc &d = pl.sd[k];
        memset(&d, 0, sizeof d);
        int n = lens[k];
        int NT = n > 0 ? (n + T - 1) / T : 0;
        int Np = NT * T;
        d.n = n;
        d.NT = NT;
        d.Np = Np;
        d.PC = round_up(Np + kColOff + 1, 8);
        d.result_index = k;
        d.code_off = (long long)o_code;  o_code += align_up((size_t)Np, 128);
        d.drow_off = (long long)o_drow;  o_drow += align_up((size_t)Np * Np, 64);
        d.dcol_off = (long long)o_dcol;  o_dcol += align_up((size_t)Np * d.PC, 64);
        if (method == kTwoVector) {
            d.rf_off = (long long)o_rf;  o_rf += align_up((size_t)Np * (Np / q), 32);
            d.cf_off = (long long)o_cf;  o_cf += align_up((size_t)(Np / q) * Np, 32);
        }
        d.flag_off = (long long)o_flag; o_flag += align_up((size_t)NT * NT, 32);
        d.cnt_off = (long long)o_cnt;   o_cnt += align_up((size_t)NT * NT, 32);
        d.p_off = (long long)o_p;       o_p += (size_t)kRing * NT * T * T;
        pl.NTs[k] = NT;
    }
    size_t off = 0;
    pl.off_control = off; off = align_up(off + 256, 256);
    pl.off_results = off; off = align_up(off + 4 * (size_t)std::max(count, 1), 256);
    pl.off_flags = off;   off = align_up(off + 4 * o_flag, 256);
    pl.off_cnt = off;     off = align_up(off + 4 * o_cnt, 256);
    pl.off_pring = off;   off = align_up(off + 4 * o_p, 256);
    pl.zero_bytes = off;
    pl.off_codes = off;   off = align_up(off + o_code, 256);
    pl.off_drow = off;    off = align_up(off + 2 * o_drow, 256);
    pl.off_dcol = off;    off = align_up(off + 2 * o_dcol, 256);
    pl.off_rf = off;      off = align_up(off + 4 * o_rf, 256);
    pl.off_cf = off;      off = align_up(off + 4 * o_cf, 256);
    pl.bytes = off;
    return pl;
}

FoldParams make_params(const fold_ctx *ctx, const Plan &pl, uint8_t *ws, const int4 *tasks, int ntasks,
                       const SeqDesc *d_sd) {
    FoldParams p;
    memset(&p, 0, sizeof p);
    p.tasks = tasks;
    p.ntasks = ntasks;
    p.queue_head = reinterpret_cast<int *>(ws + pl.off_control);
    p.error = reinterpret_cast<int *>(ws + pl.off_control) + 1;
    p.queue_head_far = reinterpret_cast<int *>(ws + pl.off_control) + 2;
    p.nnear = 0;
    p.near_ctas = 0;
    p.seqs = d_sd;
    p.codes = ws + pl.off_codes;
    p.drow = reinterpret_cast<int16_t *>(ws + pl.off_drow);
    p.dcol = reinterpret_cast<int16_t *>(ws + pl.off_dcol);
    p.rf = reinterpret_cast<uint32_t *>(ws + pl.off_rf);
    p.cf = reinterpret_cast<uint32_t *>(ws + pl.off_cf);
    p.flags = reinterpret_cast<int *>(ws + pl.off_flags);
    p.cnt = reinterpret_cast<int *>(ws + pl.off_cnt);
    p.pring = reinterpret_cast<int *>(ws + pl.off_pring);
    p.results = reinterpret_cast<int *>(ws + pl.off_results);
    p.rtab = ctx->d_rpacked;
    p.pair64 = ctx->pair64;
    p.timeout_ns = ctx->timeout_ms * 1000000LL;
    p.memo = (ctx->r_memo && ctx->method == kTwoVector) ? 1 : 0;
    return p;
}

int grid_for(fold_ctx *ctx) {
    if (ctx->grid_override > 0) return ctx->grid_override;
    int bps = fold_blocks_per_sm(ctx->q, ctx->method);
    if (bps < 1) bps = 1;
    return ctx->sm_count * bps;
}

// Work split of a single fold.  Tile tasks form the critical path (one per tile diagonal, each
// waiting for its neighbours); chunk tasks are throughput work.  Chunk warps on an SM slow the
// tile warps there (issue slots, shared memory), so tile tasks may get SMs of their own.  The
// candidate layouts, with the measured cost of one tile-diagonal step (B300, q = 8):
//   one shared queue                          about 20 us, chunks on every SM
//   tile-only CTAs taking tile tasks          about 13 us, chunks on the other SMs
//   column mode, 4 columns per tile CTA       about 9.9 us
//   column mode, 8 columns per tile CTA       about 12.5 us
// Column mode gives every tile column a warp of its own that computes it bottom-up: a tile's
// bottom neighbour is the warp's previous tile, and its left neighbour comes through shared memory
// unless it is the first column of its CTA.  A layout's time is modelled as the larger of the path
// (NT steps) and the chunk work at the measured rates (two-vector about 4.3e9 lookups per ms,
// plain about 1.77e10 split points per ms, on 148 SMs) spread over the SMs left to chunks
// (chunk-only SMs at 1/0.86 of that rate); the fastest wins.
// The options force a layout: FOLD_OPT_NEAR_CTAS (0 = one queue, k = k tile CTAs) and
// FOLD_OPT_COLUMNS (0 = no column mode, v = column mode with v columns per tile CTA).
// Size buckets of the tuned settings: four per doubling of n.
int tune_bucket(int n) { return n < 1 ? 0 : (int)std::floor(4.0 * std::log2((double)n)); }

FoldOpts single_opts(const fold_ctx *ctx, int n) {
    FoldOpts o;
    o.near_opt = ctx->near_ctas_opt;
    o.cols_opt = ctx->columns_opt;
    o.kc = ctx->kc_override;
    if (o.near_opt == -1 && o.cols_opt == -1 && o.kc == 0) {
        auto it = ctx->tune.find(tune_bucket(n));
        if (it != ctx->tune.end()) {
            o.near_opt = it->second.near_opt;
            o.cols_opt = it->second.cols_opt;
            o.kc = it->second.kc;
        }
    }
    return o;
}

SplitPlan plan_split(fold_ctx *ctx, const FoldOpts &o, int NT, int grid, bool layout_ok) {
    SplitPlan sp;
    const int nopt = o.near_opt, copt = o.cols_opt;
    if (nopt == 0 || NT < 2 || grid < 2) return sp;
    auto ceil_div = [](int a, int b) { return (a + b - 1) / b; };
    // column mode with a helper warp per column: two-vector, at most half the CTA's warps as columns;
    // automatic up to NT = 150 tiles per side (n ~ 4800 at q = 8), where it measured faster (n = 2000:
    // 0.53 against 0.61 ms, n = 4000: 1.10-1.15 against 1.19 ms); at n = 6000 the end-range chunks
    // then arrive after the tile could start and it measured slower (2.0 against 1.84 ms)
    const bool help_ok = ctx->col_helpers_opt != 0 && fold_col_helpers_supported(ctx->q, ctx->method) &&
                         (ctx->col_helpers_opt == 1 || NT <= 150);
    // finished tile CTAs joining the chunk workers: automatic without helpers, where it measured
    // faster (n = 6000 1.81 -> 1.78 ms, n = 8000 3.24 -> 3.04 ms); with helpers it measured the same
    // or up to 3 % slower (n = 2000-4000)
    auto join_for = [&](int helpers) { return ctx->col_join_opt == 1 || (ctx->col_join_opt == -1 && !helpers) ? 1 : 0; };
    auto column = [&](int cpc, int near) -> bool {
        near = std::max(near, ceil_div(NT, cpc));
        if (!layout_ok || near > grid - 1) return false;
        sp.near_ctas = near;
        sp.col_mode = 1;
        sp.cpc = cpc;
        sp.helpers = (help_ok && cpc <= kWarpsPerCta / 2) ? 1 : 0;
        sp.join = join_for(sp.helpers);
        return true;
    };
    if (nopt > 0) {                            // forced tile CTAs
        const int near = std::min(nopt, grid - 1);
        if (copt >= 1 && column(copt, near)) return sp;
        if (copt == -1 && near >= ceil_div(NT, kWarpsPerCta) && column(kWarpsPerCta, near)) return sp;
        sp.near_ctas = near;
        return sp;
    }
    if (copt >= 1) {                           // forced column mode
        column(copt, 0);
        return sp;
    }
    if (NT < 8 || grid < 12) return sp;
    const double n = (double)NT * tile_of(ctx->q, ctx->method);
    const double work_ms = (148.0 / std::max(1, ctx->sm_count)) *
                           (ctx->method == kTwoVector ? n * n * n / (6.0 * ctx->q) / 4.3e9 : n * n * n / 6.0 / 1.77e10);
    // chunk-only SMs get through their work ~1/0.86 faster than SMs that also run tiles (measured);
    // column CTAs that join the chunk workers when their columns end (the rightmost column of a CTA
    // ends after a fraction of the fold proportional to its index) count as chunk SMs half the time
    auto model = [&](double step_us, int near, bool joins = false) {
        const double held = joins ? 0.5 * near : (double)near;
        return std::max(NT * step_us * 1e-3, work_ms * grid / std::max(1.0, grid - held) * (near > 0 ? 0.86 : 1.0));
    };
    // tile-diagonal step of each layout (q = 8, measured on B300; with these figures both kernels
    // picked the fastest layout, or one within 1 %, at every size swept from n = 2000 to 16384)
    const double step_one = 20.0, step_split = 13.0;
    const double step_col[2] = {help_ok ? 8.5 : 9.9, 12.5};
    double best = model(step_one, 0);
    const int near_split = std::max(2, std::min(ceil_div(NT, kWarpsPerCta), grid / 6));
    const double split = model(step_split, near_split);
    if (split < best) {
        best = split;
        sp.near_ctas = near_split;
    }
    if (copt == 0 || !layout_ok) return sp;
    const int cands[2] = {4, 8};
    for (int k = 0; k < 2; ++k) {
        const int near = ceil_div(NT, cands[k]);
        if (near > grid / 3) continue;
        const int helpers = (help_ok && cands[k] <= kWarpsPerCta / 2) ? 1 : 0;
        const double m = model(step_col[k], near, join_for(helpers) != 0);
        if (m < best) {
            best = m;
            sp.near_ctas = near;
            sp.col_mode = 1;
            sp.cpc = cands[k];
            sp.helpers = helpers;
            sp.join = join_for(helpers);
        }
    }
    return sp;
}

// Reorders a task list into [tile tasks | chunk tasks], keeping the list order
// inside each part; returns the number of tile tasks.
int split_queues(std::vector<int4> &tasks) {
    std::vector<int4> near, far;
    near.reserve(tasks.size());
    for (const int4 &t : tasks) (task_type(t.y) == kTaskNear ? near : far).push_back(t);
    const int nn = (int)near.size();
    near.insert(near.end(), far.begin(), far.end());
    tasks.swap(near);
    return nn;
}

int status_from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return FOLD_OK;
    if (e == cudaErrorMemoryAllocation) return FOLD_ENOMEM;
    return FOLD_ECUDA;
}

// device buffer that grows on demand (context-owned)
int ensure_buf(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.ptr) return FOLD_OK;
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.ptr, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) { cudaGetLastError(); return FOLD_ENOMEM; }
    b.bytes = std::max<size_t>(bytes, 256);
    return FOLD_OK;
}

int ensure_host(HostBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.ptr) return FOLD_OK;
    if (b.ptr) cudaFreeHost(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMallocHost(&b.ptr, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) { cudaGetLastError(); return FOLD_ENOMEM; }
    b.bytes = std::max<size_t>(bytes, 256);
    return FOLD_OK;
}

// Launches the persistent kernel, with CUDA events around it when timing is
// on and a zeroed per-task trace buffer when tracing is on.
cudaError_t launch_fold_instrumented(fold_ctx *ctx, FoldParams &p, cudaStream_t st) {
    cudaError_t e;
    if (ctx->trace) {
        size_t bytes = (size_t)std::max(p.ntasks, 1) * kTraceWords * sizeof(long long);
        if (ensure_buf(ctx->trace_buf, bytes)) return cudaErrorMemoryAllocation;
        e = cudaMemsetAsync(ctx->trace_buf.ptr, 0, bytes, st);
        if (e != cudaSuccess) return e;
        p.trace = reinterpret_cast<long long *>(ctx->trace_buf.ptr);
        ctx->trace_count = p.ntasks;
    } else {
        p.trace = nullptr;
    }
    if (ctx->timing) {
        if (!ctx->ev0) {
            if ((e = cudaEventCreate(&ctx->ev0)) != cudaSuccess) return e;
            if ((e = cudaEventCreate(&ctx->ev1)) != cudaSuccess) return e;
        }
        if ((e = cudaEventRecord(ctx->ev0, st)) != cudaSuccess) return e;
    }
    e = launch_fold(p, ctx->q, ctx->method, grid_for(ctx), st);
    if (e != cudaSuccess) return e;
    if (ctx->timing) {
        if ((e = cudaEventRecord(ctx->ev1, st)) != cudaSuccess) return e;
        ctx->ev_pending = true;
    }
    return cudaSuccess;
}

// Base letters to codes; returns false on an invalid letter.
namespace {
// base -> code 0..3 (A, C, G, U in either case); every other byte -> 0x80
struct CodeTable {
    uint8_t v[256];
    CodeTable() {
        memset(v, 0x80, sizeof v);
        v['A'] = v['a'] = 0;
        v['C'] = v['c'] = 1;
        v['G'] = v['g'] = 2;
        v['U'] = v['u'] = 3;
    }
};
const CodeTable kCodes;
}  // namespace

// Device copies of task templates, at most kTemplateStoreTasks tasks (1 GiB).
constexpr size_t kTemplateStoreTasks = size_t(64) << 20;

// The first task (in ctx->tstore) of every template in tpls, uploading those not there yet; false
// when they do not fit the store (the caller then builds the list on the host).
bool dev_templates(fold_ctx *ctx, const std::vector<std::shared_ptr<const SeqTemplate>> &tpls,
                   std::vector<size_t> &first, cudaStream_t st) {
    size_t need_all = 0, need_new = 0;
    for (const auto &t : tpls) {
        need_all += t->tasks.size();
        if (!ctx->tstore_at.count(t.get())) need_new += t->tasks.size();
    }
    if (need_all > kTemplateStoreTasks) return false;
    if (need_new > 0) {
        // nothing that reads the store may still run while it is rewritten or moved
        if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return false; }
        if (ctx->tstore_used + need_new > kTemplateStoreTasks) {
            ctx->tstore_at.clear();   // start over with this batch's templates
            ctx->tstore_used = 0;
            need_new = need_all;
        }
        const size_t want = (ctx->tstore_used + need_new) * sizeof(int4);
        if (want > ctx->tstore.bytes) {
            const size_t grow = std::min(std::max(want, 2 * ctx->tstore.bytes), kTemplateStoreTasks * sizeof(int4));
            void *p = nullptr;
            if (cudaMalloc(&p, grow) != cudaSuccess) { cudaGetLastError(); return false; }
            if (ctx->tstore_used &&
                (cudaMemcpyAsync(p, ctx->tstore.ptr, ctx->tstore_used * sizeof(int4), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                 cudaStreamSynchronize(st) != cudaSuccess)) {
                cudaFree(p);
                cudaGetLastError();
                return false;
            }
            if (ctx->tstore.ptr) cudaFree(ctx->tstore.ptr);
            ctx->tstore.ptr = p;
            ctx->tstore.bytes = grow;
        }
    }
    first.resize(tpls.size());
    for (size_t k = 0; k < tpls.size(); ++k) {
        auto it = ctx->tstore_at.find(tpls[k].get());
        if (it == ctx->tstore_at.end()) {
            const size_t at = ctx->tstore_used, cnt = tpls[k]->tasks.size();
            if (cnt && cudaMemcpy(static_cast<int4 *>(ctx->tstore.ptr) + at, tpls[k]->tasks.data(), cnt * sizeof(int4),
                                  cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            ctx->tstore_used += cnt;
            it = ctx->tstore_at.emplace(tpls[k].get(), std::make_pair(tpls[k], at)).first;
        }
        first[k] = it->second.second;
    }
    return true;
}

bool encode_seq(const char *seq, int n, uint8_t *out) {
    // a table lookup per base and one check at the end: no branch that depends on the base
    unsigned bad = 0;
    for (int k = 0; k < n; ++k) {
        const uint8_t c = kCodes.v[(uint8_t)seq[k]];
        bad |= c;
        out[k] = c;
    }
    return (bad & 0x80u) == 0;
}

// Cached device schedule + descriptor for a single sequence of length n.
int single_schedule(fold_ctx *ctx, int n, const Plan &pl, const int4 **tasks, int *ntasks, int *nnear,
                    bool *layout_ok, const SeqDesc **d_sd, bool capturing) {
    int NT = pl.NTs[0];
    const FoldOpts o = single_opts(ctx, n);
    const bool drop = ctx->test_drop_task != 0;
    int kc = o.kc > 0 ? o.kc : kc_auto(NT);
    // the split list is the same for every split layout; layout_ok is assumed for the choice here
    const int nearc = plan_split(ctx, o, NT, grid_for(ctx), true).near_ctas;
    long long key = ((((long long)n << 24) | ((long long)ctx->method << 20) | ((long long)ctx->q << 16) | kc) << 12) |
                    (nearc & 0xfff);
    if (drop) key = -key - 1;   // separate cache entry for the fault-injection schedule
    std::lock_guard<std::mutex> lk(ctx->sched_mu);
    auto it = ctx->sched_cache.find(key);
    if (it == ctx->sched_cache.end()) {
        // building the list allocates and copies synchronously: not while a stream is being captured
        if (capturing) return FOLD_EINVAL;
        std::vector<int4> tv;
        build_schedule(pl.NTs, kc, strip_of(ctx->q, ctx->method), tv);
        if (drop) {
            // host-side fault injection: drop the NEAR task of tile (0,1)
            for (size_t k = 0; k < tv.size(); ++k)
                if (task_type(tv[k].y) == kTaskNear && task_I(tv[k].y) == 0 && task_J(tv[k].y) == 1) {
                    tv.erase(tv.begin() + (long)k);
                    break;
                }
        }
        CachedSched cs;
        cs.nnear = nearc > 0 ? split_queues(tv) : 0;
        cs.ntasks = (int)tv.size();
        // column mode finds tile (I, I+t) at position t*NT - t(t-1)/2 + I of the tile tasks
        cs.layout_ok = cs.nnear == NT * (NT + 1) / 2;
        for (int t = 0, k = 0; cs.layout_ok && t < NT; ++t)
            for (int I = 0; I + t < NT; ++I, ++k)
                if (tv[k].y != task_pack(kTaskNear, I, I + t)) { cs.layout_ok = false; break; }
        size_t bytes = tv.size() * sizeof(int4) + 256 + sizeof(SeqDesc);
        if (cudaMalloc(&cs.dev, bytes) != cudaSuccess) { cudaGetLastError(); return FOLD_ENOMEM; }
        cs.d_sd = reinterpret_cast<SeqDesc *>(cs.dev);
        cs.d_tasks = reinterpret_cast<int4 *>(reinterpret_cast<uint8_t *>(cs.dev) + 256);
        cudaError_t e = cudaMemcpy(cs.d_sd, pl.sd.data(), sizeof(SeqDesc), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !tv.empty())
            e = cudaMemcpy(cs.d_tasks, tv.data(), tv.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(cs.dev); return status_from_cuda(e); }
        it = ctx->sched_cache.emplace(key, cs).first;
    }
    *tasks = it->second.d_tasks;
    *ntasks = it->second.ntasks;
    *nnear = it->second.nnear;
    *layout_ok = it->second.layout_ok;
    *d_sd = it->second.d_sd;
    return FOLD_OK;
}

// Enqueues the fold of one sequence whose codes are in device memory.
// Section 4's organisation (FOLD_METHOD_SLIDING): its own workspace layout and kernel.
static int enqueue_sliding(fold_ctx *ctx, const uint8_t *d_codes, int n, uint8_t *ws, size_t ws_bytes, int32_t *d_out,
                           int16_t *d_D, cudaStream_t st) {
    const SlidingLayout L = sliding_layout(n);
    if (ws_bytes < L.bytes) return FOLD_ENOMEM;
    cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, st);
    if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(ws + L.off_drow, 0, (size_t)n * n * 2, st);
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(ws + L.off_codes, d_codes, (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    int *control = reinterpret_cast<int *>(ws + L.off_control);
    int *results = reinterpret_cast<int *>(ws + L.off_results);
    if (n >= 2) {
        SlidingParams p;
        p.codes = ws + L.off_codes;
        p.n = n;
        p.drow = reinterpret_cast<int16_t *>(ws + L.off_drow);
        p.H = reinterpret_cast<uint32_t *>(ws + L.off_H);
        p.V = reinterpret_cast<uint32_t *>(ws + L.off_V);
        p.progress = reinterpret_cast<int *>(ws + L.off_progress);
        p.next_col = control;
        p.error = control + 1;
        p.result = results;
        p.rtab = ctx->d_rpacked;
        p.pair64 = ctx->pair64;
        p.timeout_ns = ctx->timeout_ms * 1000000LL;
        if (ctx->timing) {
            if (!ctx->ev0) {
                if ((e = cudaEventCreate(&ctx->ev0)) != cudaSuccess) return status_from_cuda(e);
                if ((e = cudaEventCreate(&ctx->ev1)) != cudaSuccess) return status_from_cuda(e);
            }
            if ((e = cudaEventRecord(ctx->ev0, st)) != cudaSuccess) return status_from_cuda(e);
        }
        e = launch_sliding(p, ctx->q, ctx->sm_count, st);
        if (e == cudaSuccess && ctx->timing) {
            e = cudaEventRecord(ctx->ev1, st);
            ctx->ev_pending = true;
        }
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    e = launch_finalize(control + 1, results, 1, d_out, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    if (d_D && n > 0) {
        e = launch_extract(reinterpret_cast<int16_t *>(ws + L.off_drow), n, n, d_D, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    return FOLD_OK;
}

// Section 3.2's FG algorithm (FOLD_METHOD_FG): its own workspace layout and kernel.
static int enqueue_fg(fold_ctx *ctx, const uint8_t *d_codes, int n, uint8_t *ws, size_t ws_bytes, int32_t *d_out,
                      int16_t *d_D, cudaStream_t st) {
    const FgLayout L = fg_layout(n, ctx->q);
    if (ws_bytes < L.bytes) return FOLD_ENOMEM;
    cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, st);
    if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(ws + L.off_drow, 0, (size_t)n * n * 2, st);
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(ws + L.off_codes, d_codes, (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    int *control = reinterpret_cast<int *>(ws + L.off_control);
    int *results = reinterpret_cast<int *>(ws + L.off_results);
    if (n >= 2) {
        FgParams p;
        p.codes = ws + L.off_codes;
        p.n = n;
        p.ng = L.ng;
        p.drow = reinterpret_cast<int16_t *>(ws + L.off_drow);
        p.cv = reinterpret_cast<uint32_t *>(ws + L.off_cv);
        p.fgt = reinterpret_cast<int16_t *>(ws + L.off_fgt);
        p.progress = reinterpret_cast<int *>(ws + L.off_progress);
        p.next_col = control;
        p.error = control + 1;
        p.result = results;
        p.pair64 = ctx->pair64;
        p.timeout_ns = ctx->timeout_ms * 1000000LL;
        if (ctx->timing) {
            if (!ctx->ev0) {
                if ((e = cudaEventCreate(&ctx->ev0)) != cudaSuccess) return status_from_cuda(e);
                if ((e = cudaEventCreate(&ctx->ev1)) != cudaSuccess) return status_from_cuda(e);
            }
            if ((e = cudaEventRecord(ctx->ev0, st)) != cudaSuccess) return status_from_cuda(e);
        }
        e = launch_fg(p, ctx->q, ctx->sm_count, st);
        if (e == cudaSuccess && ctx->timing) {
            e = cudaEventRecord(ctx->ev1, st);
            ctx->ev_pending = true;
        }
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    e = launch_finalize(control + 1, results, 1, d_out, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    if (d_D && n > 0) {
        e = launch_extract(reinterpret_cast<int16_t *>(ws + L.off_drow), n, n, d_D, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    return FOLD_OK;
}

// Workspace bytes of a single fold of length n, and where its row-major table and codes sit in it.
static size_t single_bytes(const fold_ctx *ctx, int n) {
    if (ctx->method == kSliding) return sliding_layout(n).bytes;
    if (ctx->method == kFg) return fg_layout(n, ctx->q).bytes;
    return make_plan(&n, 1, ctx->q, ctx->method).bytes;
}
static void single_table(const fold_ctx *ctx, int n, uint8_t *ws, const int16_t **drow, int *stride, const uint8_t **codes) {
    if (ctx->method == kSliding) {
        const SlidingLayout L = sliding_layout(n);
        *drow = reinterpret_cast<const int16_t *>(ws + L.off_drow);
        *stride = n;
        *codes = ws + L.off_codes;
        return;
    }
    if (ctx->method == kFg) {
        const FgLayout L = fg_layout(n, ctx->q);
        *drow = reinterpret_cast<const int16_t *>(ws + L.off_drow);
        *stride = n;
        *codes = ws + L.off_codes;
        return;
    }
    Plan pl = make_plan(&n, 1, ctx->q, ctx->method);
    *drow = reinterpret_cast<const int16_t *>(ws + pl.off_drow);
    *stride = pl.sd[0].Np;
    *codes = ws + pl.off_codes;
}

int enqueue_single(fold_ctx *ctx, const uint8_t *d_codes, int n, uint8_t *ws, size_t ws_bytes, int32_t *d_out,
                   int16_t *d_D, cudaStream_t st) {
    // stream capture (CUDA graphs): only stream work may be recorded, so no allocation, timing or trace
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return FOLD_ECUDA;
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (capturing && (ctx->timing || ctx->trace)) return FOLD_EINVAL;
    if (ctx->method == kSliding) return enqueue_sliding(ctx, d_codes, n, ws, ws_bytes, d_out, d_D, st);
    if (ctx->method == kFg) return enqueue_fg(ctx, d_codes, n, ws, ws_bytes, d_out, d_D, st);
    int32_t len = n;
    Plan pl = make_plan(&len, 1, ctx->q, ctx->method);
    if (ws_bytes < pl.bytes) return FOLD_ENOMEM;
    // the task list first: a refusal leaves nothing enqueued (or recorded)
    const int4 *tasks = nullptr;
    int ntasks = 0, nnear = 0;
    bool layout_ok = false;
    const SeqDesc *d_sd = nullptr;
    if (n >= 1) {
        int rc = single_schedule(ctx, n, pl, &tasks, &ntasks, &nnear, &layout_ok, &d_sd, capturing);
        if (rc) return rc;
    }
    cudaError_t e = cudaMemsetAsync(ws, 0, pl.zero_bytes, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (n >= 1) {
        e = launch_pad_codes(d_codes, n, pl.sd[0].Np, ws + pl.off_codes, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        FoldParams p = make_params(ctx, pl, ws, tasks, ntasks, d_sd);
        if (nnear > 0) {
            const SplitPlan sp = plan_split(ctx, single_opts(ctx, n), pl.NTs[0], grid_for(ctx), layout_ok);
            p.col_mode = sp.col_mode;
            p.cols_per_cta = sp.cpc;
            p.col_helpers = sp.helpers;
            p.col_join = sp.join;
            p.nnear = nnear;
            p.near_ctas = sp.near_ctas;
        }
        e = launch_fold_instrumented(ctx, p, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 2;
    }
    e = launch_finalize(reinterpret_cast<int *>(ws + pl.off_control) + 1, reinterpret_cast<int *>(ws + pl.off_results),
                        1, d_out, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    if (d_D && n > 0) {
        e = launch_extract(reinterpret_cast<int16_t *>(ws + pl.off_drow), pl.sd[0].Np, n, d_D, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    return FOLD_OK;
}

}  // namespace fold

// ====================================================================== C-ABI
extern "C" {

const char *fold_strerror(int code) {
    switch (code) {
        case FOLD_OK: return "ok";
        case FOLD_EINVAL: return "invalid argument";
        case FOLD_ENOMEM: return "out of memory (device, host, or workspace too small)";
        case FOLD_EAGAIN: return "resource temporarily unavailable (serving budget or queue)";
        case FOLD_ETIMEOUT: return "device-side wait timed out";
        case FOLD_ECUDA: return "CUDA runtime error";
        case FOLD_ENOTREADY: return "request still in flight";
    }
    return "unknown status";
}

int fold_encode(const char *seq, int32_t n, uint8_t *codes_out) {
    if (n < 0 || n > FOLD_MAX_N || (n > 0 && (!seq || !codes_out))) return FOLD_EINVAL;
    return encode_seq(seq, n, codes_out) ? FOLD_OK : FOLD_EINVAL;
}

int fold_init(int q, uint16_t pair_mask, int device, fold_ctx **out) {
    if (!out) return FOLD_EINVAL;
    *out = nullptr;
    if (q == 0) q = 8;
    if (q < 2 || q > 10) return FOLD_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? FOLD_EINVAL : FOLD_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return FOLD_ECUDA;
    fold_ctx *ctx = new (std::nothrow) fold_ctx();
    if (!ctx) return FOLD_ENOMEM;
    ctx->device = device;
    ctx->q = q;
    ctx->pair_mask = pair_mask;
    ctx->pair64 = 0;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y)
            if ((pair_mask >> (4 * x + y)) & 1) ctx->pair64 |= 1ULL << (8 * x + y);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return FOLD_ECUDA;
    }
    size_t nent = (size_t)1 << (2 * (q - 1));
    // both copies padded to 256 bytes: the kernel stages R into shared memory in 16-byte pieces
    if (cudaMalloc(&ctx->d_rcanon, align_up(nent, 256)) != cudaSuccess ||
        cudaMalloc(&ctx->d_rpacked_buf, align_up(nent / 2, 256) + 256) != cudaSuccess) {
        cudaGetLastError();
        fold_destroy(ctx);
        return FOLD_ENOMEM;
    }
    ctx->d_rpacked = q >= 10 ? ctx->d_rpacked_buf : ctx->d_rcanon;
    cudaError_t e = launch_rtable(q, ctx->d_rcanon, ctx->d_rpacked_buf, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        fold_destroy(ctx);
        return FOLD_ECUDA;
    }
    ctx->launches = 1;
    *out = ctx;
    return FOLD_OK;
}

void fold_destroy(fold_ctx *ctx) {
    if (!ctx) return;
    fold_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->sched_cache) cudaFree(kv.second.dev);
    for (auto &kv : ctx->solo_lists) cudaFree(kv.second.dev);
    if (ctx->d_rcanon) cudaFree(ctx->d_rcanon);
    if (ctx->d_rpacked_buf) cudaFree(ctx->d_rpacked_buf);
    if (ctx->ws.ptr) cudaFree(ctx->ws.ptr);
    if (ctx->aux.ptr) cudaFree(ctx->aux.ptr);
    if (ctx->dout.ptr) cudaFree(ctx->dout.ptr);
    if (ctx->hstage.ptr) cudaFreeHost(ctx->hstage.ptr);
    if (ctx->trace_buf.ptr) cudaFree(ctx->trace_buf.ptr);
    if (ctx->tstore.ptr) cudaFree(ctx->tstore.ptr);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int fold_set_option(fold_ctx *ctx, int option, int64_t value) {
    if (!ctx) return FOLD_EINVAL;
    switch (option) {
        case FOLD_OPT_METHOD:
            if (value != FOLD_METHOD_TWO_VECTOR && value != FOLD_METHOD_PLAIN && value != FOLD_METHOD_SLIDING &&
                value != FOLD_METHOD_FG)
                return FOLD_EINVAL;
            if (ctx->serve) return FOLD_EAGAIN;   // the serving thread reads the method
            ctx->method = (int)value;
            return FOLD_OK;
        case FOLD_OPT_GRID:
            if (value < 0 || value > 1 << 20) return FOLD_EINVAL;
            ctx->grid_override = (int)value;
            return FOLD_OK;
        case FOLD_OPT_TIMEOUT_MS:
            if (value < 1 || value > 600000) return FOLD_EINVAL;
            ctx->timeout_ms = value;
            return FOLD_OK;
        case FOLD_OPT_KCHUNK:
            if (value < 0 || value > 4096) return FOLD_EINVAL;
            ctx->kc_override = (int)value;
            return FOLD_OK;
        case FOLD_OPT_TEST_DROP_TASK:
            if (value < 0 || value > 1) return FOLD_EINVAL;
            ctx->test_drop_task = (int)value;
            return FOLD_OK;
        case FOLD_OPT_TIMING:
            if (value < 0 || value > 1) return FOLD_EINVAL;
            ctx->timing = (int)value;
            return FOLD_OK;
        case FOLD_OPT_TRACE:
            if (value < 0 || value > 1) return FOLD_EINVAL;
            ctx->trace = (int)value;
            return FOLD_OK;
        case FOLD_OPT_NEAR_CTAS:
            if (value < -1 || value > 4096) return FOLD_EINVAL;
            ctx->near_ctas_opt = (int)value;
            return FOLD_OK;
        case FOLD_OPT_COLUMNS:
            if (value < -1 || value > kWarpsPerCta) return FOLD_EINVAL;
            ctx->columns_opt = (int)value;
            return FOLD_OK;
        case FOLD_OPT_COL_HELPERS:
            if (value < -1 || value > 1) return FOLD_EINVAL;
            ctx->col_helpers_opt = (int)value;
            return FOLD_OK;
        case FOLD_OPT_COL_JOIN:
            if (value < -1 || value > 1) return FOLD_EINVAL;
            ctx->col_join_opt = (int)value;
            return FOLD_OK;
        case FOLD_OPT_SERVE_RING:
            if (value < 0 || value > 1) return FOLD_EINVAL;
            if (ctx->serve) return FOLD_EAGAIN;
            ctx->serve_ring = (int)value;
            return FOLD_OK;
        case FOLD_OPT_SERVE_LONG_TILES:
            if (value < 1 || value > FOLD_MAX_N) return FOLD_EINVAL;
            if (ctx->serve) return FOLD_EAGAIN;
            ctx->serve_long_tiles = (int)value;
            return FOLD_OK;
        case FOLD_OPT_SERVE_LONG_CAP:
            if (value < 0 || value > (1 << 20)) return FOLD_EINVAL;
            if (ctx->serve) return FOLD_EAGAIN;
            ctx->serve_long_cap = (int)value;
            return FOLD_OK;
        case FOLD_OPT_BATCH_FLAT:
            if (value < -1 || value > 1) return FOLD_EINVAL;
            ctx->batch_flat_opt = (int)value;
            return FOLD_OK;
        case FOLD_OPT_BATCH_GATHER:
            if (value < 0 || value > 1) return FOLD_EINVAL;
            ctx->batch_gather = (int)value;
            return FOLD_OK;
        case FOLD_OPT_R_MEMO:
            if (value < 0 || value > 1 || (value == 1 && ctx->q >= 10)) return FOLD_EINVAL;
            if (ctx->serve) return FOLD_EAGAIN;
            ctx->r_memo = (int)value;
            return FOLD_OK;
    }
    return FOLD_EINVAL;
}

int fold_get_option(fold_ctx *ctx, int option, int64_t *value) {
    if (!ctx || !value) return FOLD_EINVAL;
    switch (option) {
        case FOLD_OPT_METHOD: *value = ctx->method; return FOLD_OK;
        case FOLD_OPT_GRID: *value = grid_for(ctx); return FOLD_OK;
        case FOLD_OPT_TIMEOUT_MS: *value = ctx->timeout_ms; return FOLD_OK;
        case FOLD_OPT_KCHUNK: *value = ctx->kc_override; return FOLD_OK;
        case FOLD_OPT_Q: *value = ctx->q; return FOLD_OK;
        case FOLD_OPT_TILE: *value = ctx->method >= kSliding ? 1 : tile_of(ctx->q, ctx->method); return FOLD_OK;
        case FOLD_OPT_LAUNCHES: *value = (int64_t)ctx->launches; return FOLD_OK;
        case FOLD_OPT_TEST_DROP_TASK: *value = ctx->test_drop_task; return FOLD_OK;
        case FOLD_OPT_TIMING: *value = ctx->timing; return FOLD_OK;
        case FOLD_OPT_TRACE: *value = ctx->trace; return FOLD_OK;
        case FOLD_OPT_NEAR_CTAS: *value = ctx->near_ctas_opt; return FOLD_OK;
        case FOLD_OPT_COLUMNS: *value = ctx->columns_opt; return FOLD_OK;
        case FOLD_OPT_COL_HELPERS: *value = ctx->col_helpers_opt; return FOLD_OK;
        case FOLD_OPT_COL_JOIN: *value = ctx->col_join_opt; return FOLD_OK;
        case FOLD_OPT_SERVE_RING: *value = ctx->serve_ring; return FOLD_OK;
        case FOLD_OPT_SERVE_LONG_TILES: *value = ctx->serve_long_tiles; return FOLD_OK;
        case FOLD_OPT_SERVE_LONG_CAP: *value = ctx->serve_long_cap; return FOLD_OK;
        case FOLD_OPT_BATCH_FLAT: *value = ctx->batch_flat_opt; return FOLD_OK;
        case FOLD_OPT_R_MEMO: *value = ctx->r_memo; return FOLD_OK;
        case FOLD_OPT_BATCH_GATHER: *value = ctx->batch_gather; return FOLD_OK;
        case FOLD_OPT_KERNEL_NS: {
            if (!ctx->ev_pending) { *value = 0; return FOLD_OK; }
            float ms = 0.f;
            cudaError_t e = cudaEventSynchronize(ctx->ev1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            if (e != cudaSuccess) return status_from_cuda(e);
            *value = (int64_t)((double)ms * 1e6);
            return FOLD_OK;
        }
    }
    return FOLD_EINVAL;
}

int64_t fold_trace_copy(fold_ctx *ctx, fold_trace_rec *out, int64_t cap) {
    if (!ctx || (!out && cap > 0) || cap < 0) return -FOLD_EINVAL;
    if (!ctx->trace_buf.ptr || ctx->trace_count == 0) return 0;
    cudaSetDevice(ctx->device);
    int64_t count = std::min<int64_t>(cap, ctx->trace_count);
    std::vector<long long> h((size_t)count * kTraceWords);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && count)
        e = cudaMemcpy(h.data(), ctx->trace_buf.ptr, (size_t)count * kTraceWords * sizeof(long long),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return -status_from_cuda(e);
    for (int64_t k = 0; k < count; ++k) {
        const long long *r = &h[(size_t)k * kTraceWords];
        fold_trace_rec &o = out[k];
        o.worker = (int32_t)(r[0] >> 32);
        o.task = (int32_t)(r[0] & 0xffffffffLL);
        o.type = (int32_t)(r[1] >> 32);
        o.seq = (int32_t)(r[1] & 0xffffffffLL);
        o.I = (int32_t)(r[2] >> 32);
        o.J = (int32_t)(r[2] & 0xffffffffLL);
        o.t_start = r[3];
        o.t_deps = r[4];
        o.t_mid = r[5];
        o.t_end = r[6];
        o.t_aux[0] = r[7];
        o.t_aux[1] = r[8];
        o.t_aux[2] = r[9];
        o.sm = (int32_t)r[10];
        o.reserved = 0;
    }
    return count;
}

int fold_schedule_check(int32_t n, int q, int method, int32_t kchunk) {
    if (n < 0 || n > FOLD_MAX_N || q < 2 || q > 10 || (method != FOLD_METHOD_TWO_VECTOR && method != FOLD_METHOD_PLAIN) ||
        kchunk < 0)
        return -FOLD_EINVAL;
    if (n == 0) return 0;
    const int T = tile_of(q, method);
    const int NT = (n + T - 1) / T;
    if (NT > 2048) return -FOLD_EINVAL;   // the check keeps NT^3 counters on the host
    const int kc = kchunk > 0 ? kchunk : kc_auto(NT);
    std::vector<int4> tv;
    std::vector<int> nts(1, NT);
    build_schedule(nts, kc, strip_of(q, method), tv);
    return check_schedule(NT, kc, strip_of(q, method), tv);
}

int fold_batch_schedule_check(int32_t count, const int32_t *lens, int q, int method, int32_t kchunk) {
    if (count < 0 || (count > 0 && !lens) || q < 2 || q > 10 ||
        (method != FOLD_METHOD_TWO_VECTOR && method != FOLD_METHOD_PLAIN) || kchunk < 0)
        return -FOLD_EINVAL;
    const int T = tile_of(q, method), strip = strip_of(q, method);
    const int kc = kchunk > 0 ? kchunk : 64;
    std::vector<int> nts((size_t)count);
    for (int k = 0; k < count; ++k) {
        if (lens[k] < 0 || lens[k] > FOLD_MAX_N) return -FOLD_EINVAL;
        nts[(size_t)k] = (lens[k] + T - 1) / T;
        if (nts[(size_t)k] > 512) return -FOLD_EINVAL;   // the check keeps NT^3 counters per size
    }
    // every distinct size's own list is valid (coverage, chunk counts, dependency order)
    std::vector<char> checked(513, 0);
    for (int v : nts) {
        if (v == 0 || checked[(size_t)v]) continue;
        checked[(size_t)v] = 1;
        const int rc = check_schedule(v, kc, strip, seq_template(v, kc, strip, false)->tasks);
        if (rc) return 10 + rc;
    }
    std::vector<int4> all;
    build_schedule(nts, kc, strip, all, false);
    // each sequence's tasks, in list order, must be its own list
    std::vector<std::vector<int4>> per((size_t)count);
    for (const int4 &t : all) {
        if (t.x < 0 || t.x >= count) return 1;
        per[(size_t)t.x].push_back(t);
    }
    for (int k = 0; k < count; ++k) {
        if (nts[(size_t)k] == 0) {
            if (!per[(size_t)k].empty()) return 2;
            continue;
        }
        const std::vector<int4> &own = seq_template(nts[(size_t)k], kc, strip, false)->tasks;
        if (own.size() != per[(size_t)k].size()) return 3;
        for (size_t e = 0; e < own.size(); ++e) {
            const int4 a = own[e], b = per[(size_t)k][e];
            if (a.y != b.y || a.z != b.z || a.w != b.w) return 4;
        }
    }
    return 0;
}

int fold_rtable(fold_ctx *ctx, uint8_t *out, int64_t cap) {
    if (!ctx || !out) return FOLD_EINVAL;
    int64_t nent = (int64_t)1 << (2 * (ctx->q - 1));
    if (cap < nent) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpy(out, ctx->d_rcanon, (size_t)nent, cudaMemcpyDeviceToHost);
    return status_from_cuda(e);
}

// Structure workspace: the fold's, then the traceback's queue of pending intervals.
static size_t structure_bytes(size_t fold_bytes, int n) {
    return align_up(fold_bytes, 256) + align_up(traceback_scratch_bytes(n), 256);
}

int64_t fold_structure_workspace_bytes(fold_ctx *ctx, int32_t n) {
    if (!ctx || n < 0 || n > FOLD_MAX_N) return -FOLD_EINVAL;
    return (int64_t)structure_bytes(single_bytes(ctx, n), n);
}

int fold_structure_dev(fold_ctx *ctx, const uint8_t *d_codes, int32_t n, void *d_ws, int64_t ws_bytes,
                       int32_t *d_max_pairs, int32_t *d_partner, void *stream) {
    if (!ctx || !d_ws || !d_max_pairs || n < 0 || n > FOLD_MAX_N || (n > 0 && (!d_codes || !d_partner)))
        return FOLD_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255) != 0) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    const size_t fold_bytes = single_bytes(ctx, n);
    if (ws_bytes < 0 || (size_t)ws_bytes < structure_bytes(fold_bytes, n)) return FOLD_ENOMEM;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *ws = reinterpret_cast<uint8_t *>(d_ws);
    int rc = enqueue_single(ctx, d_codes, n, ws, fold_bytes, d_max_pairs, nullptr, st);
    if (rc) return rc;
    if (n == 1) return status_from_cuda(cudaMemsetAsync(d_partner, 0xff, sizeof(int32_t), st));
    if (n >= 2) {
        void *scratch = ws + align_up(fold_bytes, 256);
        const int16_t *drow;
        const uint8_t *codes;
        int stride;
        single_table(ctx, n, ws, &drow, &stride, &codes);
        cudaError_t e = launch_traceback(drow, stride, codes, n, ctx->pair64, scratch, d_partner, d_max_pairs, FOLD_ECUDA,
                                         ctx->timeout_ms * 1000000LL, ctx->sm_count, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 3;   // init, parallel walk, check
    }
    return FOLD_OK;
}

int fold_structure(fold_ctx *ctx, const char *seq, int32_t n, int32_t *max_pairs, int32_t *partner_out,
                   char *dot_bracket_out) {
    if (!ctx || !max_pairs || n < 0 || n > FOLD_MAX_N || (n > 0 && !seq)) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    const size_t nn = (size_t)std::max(n, 1);
    size_t hbytes = align_up(nn, 64) + 64 + 4 * nn;
    if (ensure_host(ctx->hstage, hbytes)) return FOLD_ENOMEM;
    uint8_t *hcodes = reinterpret_cast<uint8_t *>(ctx->hstage.ptr);
    int32_t *hres = reinterpret_cast<int32_t *>(hcodes + align_up(nn, 64));
    int32_t *hpart = hres + 16;
    if (!encode_seq(seq, n, hcodes)) return FOLD_EINVAL;
    const size_t wsb = structure_bytes(single_bytes(ctx, n), n);
    size_t aux_bytes = align_up(nn, 256) + 256 + align_up(4 * nn, 256);
    if (ensure_buf(ctx->ws, wsb) || ensure_buf(ctx->aux, aux_bytes)) return FOLD_ENOMEM;
    uint8_t *dcodes = reinterpret_cast<uint8_t *>(ctx->aux.ptr);
    int32_t *dres = reinterpret_cast<int32_t *>(dcodes + align_up(nn, 256));
    int32_t *dpart = reinterpret_cast<int32_t *>(dcodes + align_up(nn, 256) + 256);
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(dcodes, hcodes, (size_t)n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    int rc = fold_structure_dev(ctx, dcodes, n, ctx->ws.ptr, (int64_t)ctx->ws.bytes, dres, dpart, st);
    if (rc) return rc;
    e = cudaMemcpyAsync(hres, dres, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(hpart, dpart, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (*hres < 0) return -*hres == FOLD_ETIMEOUT ? FOLD_ETIMEOUT : FOLD_ECUDA;
    *max_pairs = *hres;
    if (partner_out && n > 0) memcpy(partner_out, hpart, sizeof(int32_t) * (size_t)n);
    if (dot_bracket_out) {
        for (int32_t x = 0; x < n; ++x) dot_bracket_out[x] = hpart[x] < 0 ? '.' : (hpart[x] > x ? '(' : ')');
        dot_bracket_out[n] = '\0';
    }
    return FOLD_OK;
}

int64_t fold_workspace_bytes(fold_ctx *ctx, int32_t n) {
    if (!ctx || n < 0 || n > FOLD_MAX_N) return -FOLD_EINVAL;
    return (int64_t)single_bytes(ctx, n);
}

int fold_score_dev(fold_ctx *ctx, const uint8_t *d_codes, int32_t n, void *d_ws, int64_t ws_bytes,
                   int32_t *d_max_pairs, int16_t *d_D_out, void *stream) {
    if (!ctx || !d_ws || !d_max_pairs || n < 0 || n > FOLD_MAX_N || (n > 0 && !d_codes)) return FOLD_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255) != 0) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return enqueue_single(ctx, d_codes, n, reinterpret_cast<uint8_t *>(d_ws), (size_t)ws_bytes, d_max_pairs,
                          d_D_out, st);
}

int fold_score(fold_ctx *ctx, const char *seq, int32_t n, int32_t *max_pairs, int16_t *D_out) {
    if (!ctx || !max_pairs || n < 0 || n > FOLD_MAX_N || (n > 0 && !seq)) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    size_t hbytes = (size_t)std::max(n, 1) + 256;
    if (ensure_host(ctx->hstage, hbytes)) return FOLD_ENOMEM;
    uint8_t *hcodes = reinterpret_cast<uint8_t *>(ctx->hstage.ptr);
    int32_t *hres = reinterpret_cast<int32_t *>(hcodes + align_up((size_t)std::max(n, 1), 64));
    if (!encode_seq(seq, n, hcodes)) return FOLD_EINVAL;
    size_t aux_bytes = align_up((size_t)std::max(n, 1), 256) + 256;
    if (ensure_buf(ctx->ws, single_bytes(ctx, n)) || ensure_buf(ctx->aux, aux_bytes)) return FOLD_ENOMEM;
    if (D_out && n > 0 && ensure_buf(ctx->dout, (size_t)n * n * 2)) return FOLD_ENOMEM;
    uint8_t *dcodes = reinterpret_cast<uint8_t *>(ctx->aux.ptr);
    int32_t *dres = reinterpret_cast<int32_t *>(dcodes + align_up((size_t)std::max(n, 1), 256));
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(dcodes, hcodes, (size_t)n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    int rc = enqueue_single(ctx, dcodes, n, reinterpret_cast<uint8_t *>(ctx->ws.ptr), ctx->ws.bytes, dres,
                            (D_out && n > 0) ? reinterpret_cast<int16_t *>(ctx->dout.ptr) : nullptr, st);
    if (rc) return rc;
    e = cudaMemcpyAsync(hres, dres, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && D_out && n > 0)
        e = cudaMemcpyAsync(D_out, ctx->dout.ptr, (size_t)n * n * 2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (*hres < 0) return -*hres == FOLD_ETIMEOUT ? FOLD_ETIMEOUT : FOLD_ECUDA;
    *max_pairs = *hres;
    return FOLD_OK;
}

int fold_batch(fold_ctx *ctx, int32_t count, const char *const *seqs, const int32_t *lens, int32_t *max_pairs_out,
               int16_t *const *D_out) {
    if (!ctx || count < 0 || (count > 0 && (!seqs || !lens || !max_pairs_out))) return FOLD_EINVAL;
    if (ctx->method >= kSliding) return FOLD_EINVAL;   // the per-column comparison kernels fold one sequence
    if (count == 0) return FOLD_OK;
    for (int k = 0; k < count; ++k)
        if (lens[k] < 0 || lens[k] > FOLD_MAX_N || (lens[k] > 0 && !seqs[k])) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    Plan pl = make_plan(lens, count, ctx->q, ctx->method);
    cudaStream_t st = ctx->stream;
    // the workspace's zeroed part is cleared on the device while the host builds the rest
    if (ensure_buf(ctx->ws, pl.bytes)) return FOLD_ENOMEM;
    uint8_t *ws = reinterpret_cast<uint8_t *>(ctx->ws.ptr);
    cudaError_t e = cudaMemsetAsync(ws, 0, pl.zero_bytes, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    int maxNT = 0;
    for (int v : pl.NTs) maxNT = std::max(maxNT, v);
    // a batch is bound by throughput, not by one fold's critical path: chunks of kc blocks each
    // (fewer tasks) unless FOLD_OPT_BATCH_FLAT asks for the single-fold geometric sizes
    const bool flat = ctx->batch_flat_opt != 0;
    int kc = ctx->kc_override > 0 ? ctx->kc_override : (flat ? 64 : kc_auto(maxNT));
    const int strip = strip_of(ctx->q, ctx->method);
    std::vector<std::shared_ptr<const SeqTemplate>> tpls;
    std::vector<ScheduleSeg> segs;
    const size_t ntasks = schedule_segments(pl.NTs, kc, strip, !flat, tpls, segs);
    if (ntasks > (size_t)INT32_MAX) return FOLD_EINVAL;
    // the task list is gathered on the device from device copies of the per-size templates (only
    // the segment list crosses the bus) when they fit the store; else it is built here
    std::vector<size_t> tfirst;
    const bool gather = ntasks > 0 && ctx->batch_gather && dev_templates(ctx, tpls, tfirst, st);
    // host staging: codes (padded) | SeqDesc | segments or tasks | results
    size_t codes_bytes = pl.off_drow - pl.off_codes;
    size_t sd_bytes = align_up(sizeof(SeqDesc) * count, 256);
    size_t task_bytes = align_up(ntasks * sizeof(int4), 256);
    size_t res_bytes = align_up(4 * (size_t)count, 256);
    const size_t seg_bytes = gather ? align_up(segs.size() * sizeof(int4), 256) : 0;
    const size_t list_bytes = gather ? seg_bytes : task_bytes;
    if (ensure_host(ctx->hstage, codes_bytes + sd_bytes + list_bytes + res_bytes)) return FOLD_ENOMEM;
    uint8_t *h = reinterpret_cast<uint8_t *>(ctx->hstage.ptr);
    uint8_t *hcodes = h;
    {
        // each sequence's codes, then its padding up to the next one's (a few threads for big batches)
        std::vector<size_t> code_end((size_t)count);
        for (int k = 0; k < count; ++k)
            code_end[(size_t)k] = k + 1 < count ? (size_t)pl.sd[(size_t)k + 1].code_off : codes_bytes;
        if (count > 0 && pl.sd[0].code_off > 0) memset(hcodes, kPadCode, (size_t)pl.sd[0].code_off);
        std::vector<char> ok((size_t)count, 1);
        auto enc = [&](int k0, int k1) {
            for (int k = k0; k < k1; ++k) {
                uint8_t *o = hcodes + pl.sd[(size_t)k].code_off;
                ok[(size_t)k] = encode_seq(seqs[k], lens[k], o);
                memset(o + lens[k], kPadCode, code_end[(size_t)k] - (size_t)pl.sd[(size_t)k].code_off - (size_t)lens[k]);
            }
        };
        const size_t bases = codes_bytes;
        const int nth = bases < (size_t(1) << 21) ? 1 : (int)std::min<unsigned>(8u, std::max(1u, std::thread::hardware_concurrency()));
        if (nth == 1) {
            enc(0, count);
        } else {
            std::vector<std::thread> th;
            for (int w = 0; w < nth; ++w) th.emplace_back(enc, (int)((long long)count * w / nth), (int)((long long)count * (w + 1) / nth));
            for (auto &x : th) x.join();
        }
        for (int k = 0; k < count; ++k)
            if (!ok[(size_t)k]) return FOLD_EINVAL;
    }
    memcpy(h + codes_bytes, pl.sd.data(), sizeof(SeqDesc) * count);
    int4 *hlist = reinterpret_cast<int4 *>(h + codes_bytes + sd_bytes);
    if (gather) {
        for (size_t k = 0; k < segs.size(); ++k) {
            const ScheduleSeg &sg = segs[k];
            hlist[k] = make_int4((int)(tfirst[(size_t)sg.tpl] + (size_t)sg.first), sg.count, sg.seq, (int)sg.dst);
        }
    } else {
        build_schedule_into(pl.NTs, kc, strip, !flat, hlist, ntasks);
    }
    int32_t *hres = reinterpret_cast<int32_t *>(h + codes_bytes + sd_bytes + list_bytes);
    if (ensure_buf(ctx->aux, sd_bytes + task_bytes + res_bytes + seg_bytes)) return FOLD_ENOMEM;
    uint8_t *aux = reinterpret_cast<uint8_t *>(ctx->aux.ptr);
    SeqDesc *d_sd = reinterpret_cast<SeqDesc *>(aux);
    int4 *d_tasks = reinterpret_cast<int4 *>(aux + sd_bytes);
    int32_t *d_res = reinterpret_cast<int32_t *>(aux + sd_bytes + task_bytes);
    int4 *d_segs = reinterpret_cast<int4 *>(aux + sd_bytes + task_bytes + res_bytes);
    e = cudaMemcpyAsync(ws + pl.off_codes, hcodes, codes_bytes, cudaMemcpyHostToDevice, st);
    if (gather) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(aux, h + codes_bytes, sd_bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_segs, hlist, segs.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = launch_gather_tasks(static_cast<const int4 *>(ctx->tstore.ptr), d_segs, (int)segs.size(), d_tasks,
                                    ctx->sm_count, st);
        if (e == cudaSuccess) ctx->launches += 1;
    } else if (e == cudaSuccess) {
        e = cudaMemcpyAsync(aux, h + codes_bytes, sd_bytes + task_bytes, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return status_from_cuda(e);
    FoldParams p = make_params(ctx, pl, ws, d_tasks, (int)ntasks, d_sd);
    if (ntasks > 0) {
        e = launch_fold_instrumented(ctx, p, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    e = launch_finalize(p.error, p.results, count, d_res, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    e = cudaMemcpyAsync(hres, d_res, 4 * (size_t)count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return status_from_cuda(e);
    int status = FOLD_OK;
    for (int k = 0; k < count; ++k) {
        if (hres[k] < 0) status = -hres[k] == FOLD_ETIMEOUT ? FOLD_ETIMEOUT : FOLD_ECUDA;
        max_pairs_out[k] = lens[k] >= 2 ? hres[k] : 0;
    }
    if (status) return status;
    if (D_out) {
        for (int k = 0; k < count; ++k) {
            int n = lens[k];
            if (!D_out[k] || n == 0) continue;
            if (ensure_buf(ctx->dout, (size_t)n * n * 2)) return FOLD_ENOMEM;
            e = launch_extract(p.drow + pl.sd[k].drow_off, pl.sd[k].Np, n, reinterpret_cast<int16_t *>(ctx->dout.ptr), st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(D_out[k], ctx->dout.ptr, (size_t)n * n * 2, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return status_from_cuda(e);
            ctx->launches += 1;
        }
    }
    return FOLD_OK;
}

}  // extern "C"
