// batch_graph.cu -- a batch folded in one persistent launch from caller device buffers, with a host
// plan made once: the enqueue allocates nothing, copies nothing from the host and never waits, so
// it can be recorded into a CUDA graph by stream capture and replayed on new inputs.
//
// fold_batch (api.cu) encodes host strings, builds the interleaved task list and waits for the
// answers; for a fixed set of lengths everything but the codes is the same from call to call.  The
// plan holds that part on the device: the sequences' descriptors (workspace layout), the task list
// of the one persistent launch (every sequence's list step by step, as fold_batch builds it) and
// each sequence's offset in the caller's concatenated codes.  fold_batch_dev then enqueues: clear
// the workspace's control part, scatter the codes into each sequence's padded slot, the persistent
// fold kernel (Section 4 wavefront per sequence, two-vector or plain as the context's method), and
// the answers D(0, n_k - 1) into a caller device array.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "api_internal.h"
#include "fold.h"
#include "fold_common.h"
#include "kernels.h"
#include "schedule.h"

struct fold_batch_plan {
    fold_ctx *ctx = nullptr;
    int q = 0, method = 0, count = 0, ntasks = 0;
    fold::Plan pl;
    void *dev = nullptr;                 // [SeqDesc x count | tasks | source offsets]
    fold::SeqDesc *d_sd = nullptr;
    int4 *d_tasks = nullptr;
    long long *d_src = nullptr;          // offset of sequence k's codes in the concatenated input
    long long total = 0;                 // sum of the lengths
};

namespace fold {
namespace {

// Sequence k's codes from the concatenated input into its padded slot (padding pairs with nothing).
__global__ void scatter_codes_kernel(const uint8_t *__restrict__ cat, const SeqDesc *__restrict__ sd,
                                     const long long *__restrict__ src, int count, uint8_t *__restrict__ codes) {
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        const SeqDesc d = sd[k];
        const uint8_t *in = cat + src[k];
        uint8_t *out = codes + d.code_off;
        for (int e = threadIdx.x; e < d.Np; e += blockDim.x) out[e] = e < d.n ? in[e] : (uint8_t)kPadCode;
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace fold

using namespace fold;

extern "C" {

int fold_batch_plan_create(fold_ctx *ctx, int32_t count, const int32_t *lens, fold_batch_plan **out) {
    if (!out) return FOLD_EINVAL;
    *out = nullptr;
    if (!ctx || count < 1 || !lens) return FOLD_EINVAL;
    if (ctx->method >= kSliding) return FOLD_EINVAL;   // the per-column comparison kernels fold one sequence
    long long total = 0;
    for (int k = 0; k < count; ++k) {
        if (lens[k] < 0 || lens[k] > FOLD_MAX_N) return FOLD_EINVAL;
        total += lens[k];
    }
    cudaSetDevice(ctx->device);
    fold_batch_plan *bp = new fold_batch_plan;
    bp->ctx = ctx;
    bp->q = ctx->q;
    bp->method = ctx->method;
    bp->count = count;
    bp->total = total;
    bp->pl = make_plan(lens, count, ctx->q, ctx->method);
    int maxNT = 0;
    for (int v : bp->pl.NTs) maxNT = std::max(maxNT, v);
    // the same list as fold_batch: fixed chunks of kc blocks unless FOLD_OPT_BATCH_FLAT asks for the
    // single fold's geometric sizes
    const bool flat = ctx->batch_flat_opt != 0;
    const int kc = ctx->kc_override > 0 ? ctx->kc_override : (flat ? 64 : kc_auto(maxNT));
    const size_t ntasks = build_schedule_into(bp->pl.NTs, kc, strip_of(ctx->q, ctx->method), !flat, nullptr, 0);
    if (ntasks > (size_t)INT32_MAX) {
        delete bp;
        return FOLD_EINVAL;
    }
    std::vector<int4> tasks(ntasks);
    if (ntasks) build_schedule_into(bp->pl.NTs, kc, strip_of(ctx->q, ctx->method), !flat, tasks.data(), ntasks);
    std::vector<long long> src((size_t)count);
    long long o = 0;
    for (int k = 0; k < count; ++k) {
        src[(size_t)k] = o;
        o += lens[k];
    }
    const size_t sd_bytes = align256(sizeof(SeqDesc) * count);
    const size_t task_bytes = align256(sizeof(int4) * std::max<size_t>(ntasks, 1));
    const size_t src_bytes = align256(sizeof(long long) * count);
    if (cudaMalloc(&bp->dev, sd_bytes + task_bytes + src_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete bp;
        return FOLD_ENOMEM;
    }
    uint8_t *d = reinterpret_cast<uint8_t *>(bp->dev);
    bp->d_sd = reinterpret_cast<SeqDesc *>(d);
    bp->d_tasks = reinterpret_cast<int4 *>(d + sd_bytes);
    bp->d_src = reinterpret_cast<long long *>(d + sd_bytes + task_bytes);
    bp->ntasks = (int)ntasks;
    cudaError_t e = cudaMemcpy(bp->d_sd, bp->pl.sd.data(), sizeof(SeqDesc) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ntasks) e = cudaMemcpy(bp->d_tasks, tasks.data(), sizeof(int4) * ntasks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bp->d_src, src.data(), sizeof(long long) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(bp->dev);
        delete bp;
        return status_from_cuda(e);
    }
    *out = bp;
    return FOLD_OK;
}

int64_t fold_batch_plan_workspace_bytes(const fold_batch_plan *plan) {
    if (!plan) return -FOLD_EINVAL;
    return (int64_t)plan->pl.bytes;
}

int64_t fold_batch_plan_codes_bytes(const fold_batch_plan *plan) {
    if (!plan) return -FOLD_EINVAL;
    return (int64_t)plan->total;
}

void fold_batch_plan_destroy(fold_batch_plan *plan) {
    if (!plan) return;
    if (plan->ctx) {
        cudaSetDevice(plan->ctx->device);
        cudaDeviceSynchronize();   // no enqueued fold of this plan may still read its lists
    }
    if (plan->dev) cudaFree(plan->dev);
    delete plan;
}

int fold_batch_dev(fold_ctx *ctx, const fold_batch_plan *plan, const uint8_t *d_codes, void *d_ws, int64_t ws_bytes,
                   int32_t *d_max_pairs, void *stream) {
    if (!ctx || !plan || plan->ctx != ctx || !d_ws || !d_max_pairs || (plan->total > 0 && !d_codes)) return FOLD_EINVAL;
    if (plan->q != ctx->q || plan->method != ctx->method) return FOLD_EINVAL;   // planned for another method or q
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255) != 0) return FOLD_EINVAL;
    if (ws_bytes < (int64_t)plan->pl.bytes) return FOLD_ENOMEM;
    cudaSetDevice(ctx->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return FOLD_ECUDA;
    // kernel timing and tracing record host-side state per launch: not while a graph is recorded
    if (cap != cudaStreamCaptureStatusNone && (ctx->timing || ctx->trace)) return FOLD_EINVAL;
    uint8_t *ws = reinterpret_cast<uint8_t *>(d_ws);
    const Plan &pl = plan->pl;
    cudaError_t e = cudaMemsetAsync(ws, 0, pl.zero_bytes, st);   // control, results, flags, counters, P ring
    if (e != cudaSuccess) return status_from_cuda(e);
    const int blocks = std::max(1, std::min(plan->count, 8 * std::max(ctx->sm_count, 1)));
    scatter_codes_kernel<<<blocks, 256, 0, st>>>(d_codes, plan->d_sd, plan->d_src, plan->count, ws + pl.off_codes);
    e = cudaGetLastError();
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    FoldParams p = make_params(ctx, pl, ws, plan->d_tasks, plan->ntasks, plan->d_sd);
    if (plan->ntasks > 0) {
        e = launch_fold_instrumented(ctx, p, st);
        if (e != cudaSuccess) return status_from_cuda(e);
        ctx->launches += 1;
    }
    e = launch_finalize(p.error, p.results, plan->count, d_max_pairs, st);
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    return FOLD_OK;
}

int fold_batch_dev_table(fold_ctx *ctx, const fold_batch_plan *plan, const void *d_ws, int32_t k, int16_t *d_D_out,
                         void *stream) {
    if (!ctx || !plan || plan->ctx != ctx || !d_ws || k < 0 || k >= plan->count) return FOLD_EINVAL;
    const int n = plan->pl.sd[(size_t)k].n;
    if (n == 0) return FOLD_OK;
    if (!d_D_out) return FOLD_EINVAL;
    cudaSetDevice(ctx->device);
    const Plan &pl = plan->pl;
    const int16_t *drow = reinterpret_cast<const int16_t *>(reinterpret_cast<const uint8_t *>(d_ws) + pl.off_drow) +
                          pl.sd[(size_t)k].drow_off;
    cudaError_t e = launch_extract(drow, pl.sd[(size_t)k].Np, n, d_D_out, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return status_from_cuda(e);
    ctx->launches += 1;
    return FOLD_OK;
}

}  // extern "C"
