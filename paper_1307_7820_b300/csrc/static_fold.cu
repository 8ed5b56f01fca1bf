// static_fold.cu -- fold entry point that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc when they fold -- for
// example code running inside a framework that owns all device memory
// through its own allocator and forbids allocations it does not see, service
// processes that allocate everything at start-up and must not allocate (or
// implicitly synchronise the device, as cudaMalloc/cudaFree can) on the
// request path, and plugins or callbacks that run where allocation is not
// permitted.  fold_score_static needs neither a context nor a workspace: its
// scratch (DP tables, difference vectors, tile flags, the task lists and the
// R table) lives in one file-scope __device__ array of kStaticBytes, which
// every GPU that loads this library holds until the process exits.  The
// caller passes only inputs and outputs.
//
// Limits and rules: two-vector method with q = 8; n <= FOLD_STATIC_MAX_N
// (larger n is rejected with FOLD_EINVAL).  Every call uses the same array, so
// calls that overlap on the GPU (on different streams, or from different
// threads) race and corrupt each other's results; serialise them.  The first
// call on a device does the set-up for that device (looks up the array's
// device address, builds the R table and uploads the task list of every tile
// count up to FOLD_STATIC_MAX_N / 32, then synchronises the stream), so make
// that first call before any stream capture.  After it a call only enqueues
// a memset and kernel launches: the sequence descriptor travels as a kernel
// argument and the task list is already on the device, so no host memory is
// read by the GPU.  The set-up is not redone after cudaDeviceReset.
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

constexpr int kStaticT = tile_of(kStaticQ, kTwoVector);
constexpr int kStaticMaxNT = (FOLD_STATIC_MAX_N + kStaticT - 1) / kStaticT;

// Scratch layout: R (canonical and packed, 2 x 16 KiB) | the sequence descriptor | the task lists of
// NT = 1 .. kStaticMaxNT tiles per side | the workspace of the current call (its plan).
constexpr size_t kStaticSdOff = 2 * kStaticRBytes;
constexpr size_t kStaticTasksOff = kStaticSdOff + 256;

struct StaticDevice {
    bool ready = false;
    uint8_t *base = nullptr;     // device address of g_fold_static_scratch on this device
    int sm_count = 1;
    int blocks_per_sm = 1;
    size_t task_first[kStaticMaxNT + 1] = {};   // first task of the list of NT tiles (in int4)
    int task_count[kStaticMaxNT + 1] = {};
    size_t ws_off = 0;                          // byte offset of the call's workspace
};
static StaticDevice g_static_dev[kStaticMaxDevices];
static std::mutex g_static_mu;

static size_t st_align(size_t v) { return (v + 255) / 256 * 256; }

// The sequence descriptor reaches the device as a kernel argument, so a call reads no host memory.
__global__ void static_desc_kernel(SeqDesc sd, SeqDesc *dst) { *dst = sd; }

// Per-device set-up: device address of the scratch, the R table and every task list in it.
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
        // the task list depends only on the tile count: build all of them once, in one host buffer
        std::vector<int4> all, one;
        for (int NT = 1; NT <= kStaticMaxNT; ++NT) {
            one.clear();
            build_schedule(std::vector<int>{NT}, kc_auto(NT), strip_of(kStaticQ, kTwoVector), one);
            sd.task_first[NT] = all.size();
            sd.task_count[NT] = (int)one.size();
            all.insert(all.end(), one.begin(), one.end());
        }
        sd.ws_off = st_align(kStaticTasksOff + all.size() * sizeof(int4));
        int32_t nmax = FOLD_STATIC_MAX_N;
        if (sd.ws_off + make_plan(&nmax, 1, kStaticQ, kTwoVector).bytes > kStaticBytes) return FOLD_ENOMEM;
        // R sits at the start of the scratch; q = 8 uses the byte table directly
        e = launch_rtable(kStaticQ, sd.base, sd.base + kStaticRBytes, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sd.base + kStaticTasksOff, all.data(), all.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // `all` is freed on return
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

    int32_t len = n;
    Plan pl = make_plan(&len, 1, kStaticQ, kTwoVector);
    const int NT = pl.NTs[0];
    if (sdv->ws_off + pl.bytes > kStaticBytes) return FOLD_EINVAL;   // checked at set-up for the largest n
    uint8_t *base = sdv->base;
    uint8_t *ws = base + sdv->ws_off;

    unsigned long long pair64 = 0;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y)
            if ((pair_mask >> (4 * x + y)) & 1) pair64 |= 1ULL << (8 * x + y);

    cudaError_t e = cudaMemsetAsync(ws, 0, pl.zero_bytes, st);   // control, flags, counters, partial maxima
    if (e == cudaSuccess && n > 0) {
        SeqDesc *d_sd = reinterpret_cast<SeqDesc *>(base + kStaticSdOff);
        static_desc_kernel<<<1, 1, 0, st>>>(pl.sd[0], d_sd);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_pad_codes(d_codes, n, pl.sd[0].Np, ws + pl.off_codes, st);
        FoldParams p;
        memset(&p, 0, sizeof p);
        p.tasks = reinterpret_cast<const int4 *>(base + kStaticTasksOff) + sdv->task_first[NT];
        p.ntasks = sdv->task_count[NT];
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
