// api_internal.h -- context and planning structures shared by api.cu and
// serve.cu (internal to libfold_b300).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "fold_common.h"
#include "schedule.h"

namespace fold {

struct DevBuf { void *ptr = nullptr; size_t bytes = 0; };
struct HostBuf { void *ptr = nullptr; size_t bytes = 0; };

// A lone serving request's task list on the device (see fold_ctx::solo_lists).
struct SoloList {
    void *dev = nullptr;
    size_t bytes = 0;
    int ntasks = 0, nnear = 0;
    unsigned long long used = 0;
};

struct CachedSched {
    void *dev = nullptr;
    SeqDesc *d_sd = nullptr;
    int4 *d_tasks = nullptr;
    int ntasks = 0;
    int nnear = 0;             // > 0: tasks are split [tile tasks | chunk tasks]
    bool layout_ok = false;    // the tile tasks are in diagonal order, every tile once (column mode)
};

// Workspace layout of a set of sequences (byte offsets into one buffer).
struct Plan {
    int q = 8, method = 0, T = 32, count = 0;
    std::vector<SeqDesc> sd;
    std::vector<int> NTs;
    size_t off_control = 0, off_results = 0, off_flags = 0, off_cnt = 0, off_pring = 0;
    size_t off_codes = 0, off_drow = 0, off_dcol = 0, off_rf = 0, off_cf = 0;
    size_t zero_bytes = 0, bytes = 0;
};

struct ServeState;  // serve.cu

}  // namespace fold

namespace fold {
struct TuneEntry {
    int near_opt = -1;   // FOLD_OPT_NEAR_CTAS value
    int cols_opt = -1;   // FOLD_OPT_COLUMNS value
    int kc = 0;          // FOLD_OPT_KCHUNK value (0: automatic)
    float ms = 0.f;      // measured fold time
};
// Settings a single fold of one size runs with: the options if any is set, else the tuned entry
// of the size's bucket, else automatic.
struct FoldOpts {
    int near_opt = -1, cols_opt = -1, kc = 0;
};
int tune_bucket(int n);
}  // namespace fold

struct fold_ctx {
    int device = 0;
    int q = 8;
    int method = 0;
    uint16_t pair_mask = 0;
    unsigned long long pair64 = 0;
    int sm_count = 1;
    int grid_override = 0;
    int kc_override = 0;
    long long timeout_ms = 5000;
    int test_drop_task = 0;
    int near_ctas_opt = -1;    // -1 automatic, 0 one shared queue, k > 0 k tile-only CTAs
    int columns_opt = -1;      // -1 automatic, 0 off, v >= 1 column mode with v columns per tile CTA
    int col_helpers_opt = -1;  // FOLD_OPT_COL_HELPERS: -1 automatic, 0 off, 1 on (column mode, two-vector)
    int col_join_opt = -1;     // FOLD_OPT_COL_JOIN: -1 automatic (without helpers), 0 off, 1 on
    int serve_ring = 1;        // FOLD_OPT_SERVE_RING: serving through one persistent launch fed while it runs
    int serve_long_tiles = 160;   // FOLD_OPT_SERVE_LONG_TILES: a request this many tiles per side is long
    int serve_long_cap = 2;       // FOLD_OPT_SERVE_LONG_CAP: long requests in flight at once (0: no cap)
    int batch_flat_opt = -1;   // fold_batch chunks: -1 / 1 kc blocks each, 0 geometric sizes
    int batch_gather = 1;      // FOLD_OPT_BATCH_GATHER: fold_batch's list gathered on the device
    int r_memo = 0;            // FOLD_OPT_R_MEMO: tabulate R rows on first sight (two-vector, q <= 9)
    // tuned single-fold settings per size bucket (fold_tune / fold_tune_load); used when no option
    // forces a layout or a chunk size
    std::map<int, fold::TuneEntry> tune;
    cudaStream_t stream = nullptr;
    uint8_t *d_rcanon = nullptr;
    uint8_t *d_rpacked_buf = nullptr;
    const uint8_t *d_rpacked = nullptr;
    std::map<long long, fold::CachedSched> sched_cache;   // guarded by sched_mu
    std::mutex sched_mu;
    fold::DevBuf ws, aux, dout;
    fold::HostBuf hstage;
    // device copies of the task templates fold_batch gathers its list from: the templates (held, so
    // each stays the same object) and the index of their first task in tstore
    fold::DevBuf tstore;
    size_t tstore_used = 0;
    std::map<const fold::SeqTemplate *, std::pair<std::shared_ptr<const fold::SeqTemplate>, size_t>> tstore_at;
    unsigned long long launches = 0;
    // kernel timing (FOLD_OPT_TIMING) and task tracing (FOLD_OPT_TRACE)
    int timing = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ev_pending = false;
    int trace = 0;
    fold::DevBuf trace_buf;
    int trace_count = 0;
    fold::ServeState *serve = nullptr;
    // serving: the task lists of lone requests (folded with the single fold's work split) on the
    // device per (tiles per side, chunk size, split into tile and chunk queues), built at first use
    // or ahead by fold_serve_warm, kept for the context's life (least recently used dropped past
    // 256 MiB)
    std::map<std::tuple<int, int, bool>, fold::SoloList> solo_lists;   // guarded by solo_mu
    std::mutex solo_mu;
    size_t solo_list_bytes = 0;
    unsigned long long solo_clock = 0;
};

namespace fold {
Plan make_plan(const int32_t *lens, int count, int q, int method);
FoldParams make_params(const fold_ctx *ctx, const Plan &pl, uint8_t *ws, const int4 *tasks, int ntasks,
                       const SeqDesc *d_sd);
int grid_for(fold_ctx *ctx);
int kc_auto(int NT);
int status_from_cuda(cudaError_t e);
cudaError_t launch_fold_instrumented(fold_ctx *ctx, FoldParams &p, cudaStream_t st);
struct SplitPlan {
    int near_ctas = 0;   // tile-only CTAs (0: one shared queue)
    int col_mode = 0;    // 1: column mode
    int cpc = kWarpsPerCta;   // columns per tile CTA in column mode
    int helpers = 0;     // 1: column mode with a helper warp per column (cpc <= kWarpsPerCta / 2)
    int join = 0;        // 1: column mode, a tile CTA's warps take chunks once its columns are done
};
SplitPlan plan_split(fold_ctx *ctx, const FoldOpts &o, int NT, int grid, bool layout_ok);
FoldOpts single_opts(const fold_ctx *ctx, int n);
int enqueue_single(fold_ctx *ctx, const uint8_t *d_codes, int n, uint8_t *ws, size_t ws_bytes, int32_t *d_out,
                   int16_t *d_D, cudaStream_t st);
int split_queues(std::vector<int4> &tasks);
bool encode_seq(const char *seq, int n, uint8_t *out);

int ensure_buf(DevBuf &b, size_t bytes);
int ensure_host(HostBuf &b, size_t bytes);
}  // namespace fold
