// static_fold.cu -- fold entry point that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc when they fold -- for
// example code running inside a framework that owns all device memory
// through its own allocator and forbids allocations it does not see, service
// processes that allocate everything at start-up and must not allocate (or
// implicitly synchronise the device, as cudaMalloc/cudaFree can) on the
// request path, and plugins or callbacks that run where allocation is not
// permitted.  fold_score_static needs neither a context nor a workspace: its
// scratch (DP tables, difference vectors, tile flags, the task list and the R
// table) lives in one file-scope __device__ array of kStaticBytes, which every
// GPU that loads this library holds until the process exits.  The caller
// passes only inputs and outputs.
//
// Limits and rules: two-vector method with q = 8; n <= FOLD_STATIC_MAX_N
// (larger n is rejected with FOLD_EINVAL).  Every call uses the same array, so
// calls that overlap on the GPU (on different streams, or from different
// threads) race and corrupt each other's results; serialise them.  The first
// call on a device does the set-up for that device (looks up the array's
// device address and builds the R table, then synchronises the stream), so
// make that first call before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "api_internal.h"
#include "fold.h"
#include "fold_common.h"
#include "kernels.h"
#include "schedule.h"

namespace fold {

constexpr size_t kStaticBytes = 8u << 20;   // fits a q = 8 fold of up to FOLD_STATIC_MAX_N bases
constexpr int kStaticQ = 8;
constexpr int kStaticMaxDevices = 64;
constexpr size_t kStaticRBytes = 1u << (2 * (kStaticQ - 1));   // 16 KiB

// The scratch.  In host code this name is only a stand-in for the symbol, not
// a device address: kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_fold_static_scratch[kStaticBytes];

struct StaticDevice {
    bool ready = false;
    uint8_t *base = nullptr;     // device address of g_fold_static_scratch on this device
    int sm_count = 1;
    int blocks_per_sm = 1;
};
static StaticDevice g_static_dev[kStaticMaxDevices];
static std::mutex g_static_mu;

static size_t st_align(size_t v) { return (v + 255) / 256 * 256; }

// Per-device set-up: device address of the scratch and the R table in it.
static int static_setup(int dev, cudaStream_t st, StaticDevice **out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice &sd = g_static_dev[dev];
    if (!sd.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fold_static_scratch);
        if (e != cudaSuccess || !p) return FOLD_ECUDA;
        sd.base = reinterpret_cast<uint8_t *>(p);
        cudaDeviceGetAttribute(&sd.sm_count, cudaDevAttrMultiProcessorCount, dev);
        sd.blocks_per_sm = fold_blocks_per_sm(kStaticQ, kTwoVector);
        if (sd.blocks_per_sm < 1) sd.blocks_per_sm = 1;
        // R sits at the start of the scratch; q = 8 uses the byte table directly
        e = launch_rtable(kStaticQ, sd.base, sd.base + kStaticRBytes, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return FOLD_ECUDA;
        sd.ready = true;
    }
    *out = &sd;
    return FOLD_OK;
}

}  // namespace fold

using namespace fold;

extern "C" int fold_score_static(const uint8_t *d_codes, int32_t n, uint16_t pair_mask, int32_t *d_max_pairs,
                                 int16_t *d_D_out, void *stream) {
    if (!d_max_pairs || n < 0 || n > FOLD_STATIC_MAX_N || (n > 0 && !d_codes)) return FOLD_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return FOLD_ECUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    StaticDevice *sdv = nullptr;
    int rc = static_setup(dev, st, &sdv);
    if (rc) return rc;

    // layout inside the scratch: R (2 x 16 KiB) | descriptor | tasks | the single-sequence plan
    int32_t len = n;
    Plan pl = make_plan(&len, 1, kStaticQ, kTwoVector);
    std::vector<int4> tasks;
    if (n > 0) build_schedule(pl.NTs, kc_auto(pl.NTs[0]), strip_of(kStaticQ, kTwoVector), tasks);
    const size_t o_sd = 2 * kStaticRBytes;
    const size_t o_tasks = st_align(o_sd + sizeof(SeqDesc));
    const size_t o_plan = st_align(o_tasks + tasks.size() * sizeof(int4));
    if (o_plan + pl.bytes > kStaticBytes) return FOLD_EINVAL;   // cannot happen for n <= FOLD_STATIC_MAX_N
    uint8_t *base = sdv->base;
    uint8_t *ws = base + o_plan;

    unsigned long long pair64 = 0;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y)
            if ((pair_mask >> (4 * x + y)) & 1) pair64 |= 1ULL << (8 * x + y);

    cudaError_t e = cudaMemsetAsync(ws, 0, pl.zero_bytes, st);   // control, flags, counters, partial maxima
    if (e == cudaSuccess && n > 0) {
        e = cudaMemcpyAsync(base + o_sd, pl.sd.data(), sizeof(SeqDesc), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + o_tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_pad_codes(d_codes, n, pl.sd[0].Np, ws + pl.off_codes, st);
        FoldParams p;
        memset(&p, 0, sizeof p);
        p.tasks = reinterpret_cast<const int4 *>(base + o_tasks);
        p.ntasks = (int)tasks.size();
        p.queue_head = reinterpret_cast<int *>(ws + pl.off_control);
        p.error = reinterpret_cast<int *>(ws + pl.off_control) + 1;
        p.queue_head_far = reinterpret_cast<int *>(ws + pl.off_control) + 2;
        p.nnear = 0;
        p.near_ctas = 0;
        p.seqs = reinterpret_cast<const SeqDesc *>(base + o_sd);
        p.codes = ws + pl.off_codes;
        p.drow = reinterpret_cast<int16_t *>(ws + pl.off_drow);
        p.dcol = reinterpret_cast<int16_t *>(ws + pl.off_dcol);
        p.rf = reinterpret_cast<uint32_t *>(ws + pl.off_rf);
        p.cf = reinterpret_cast<uint32_t *>(ws + pl.off_cf);
        p.flags = reinterpret_cast<int *>(ws + pl.off_flags);
        p.cnt = reinterpret_cast<int *>(ws + pl.off_cnt);
        p.pring = reinterpret_cast<int *>(ws + pl.off_pring);
        p.results = reinterpret_cast<int *>(ws + pl.off_results);
        p.rtab = base;
        p.pair64 = pair64;
        p.timeout_ns = 5000LL * 1000000LL;
        p.trace = nullptr;
        if (e == cudaSuccess) e = launch_fold(p, kStaticQ, kTwoVector, sdv->sm_count * sdv->blocks_per_sm, st);
    }
    if (e == cudaSuccess)
        e = launch_finalize(reinterpret_cast<int *>(ws + pl.off_control) + 1, reinterpret_cast<int *>(ws + pl.off_results),
                            1, d_max_pairs, st);
    if (e == cudaSuccess && d_D_out && n > 0)
        e = launch_extract(reinterpret_cast<int16_t *>(ws + pl.off_drow), pl.sd[0].Np, n, d_D_out, st);
    return e == cudaSuccess ? FOLD_OK : FOLD_ECUDA;
}
