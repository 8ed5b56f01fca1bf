// lookup_bench.cu -- attainable rate of R-table lookups in shared memory on this GPU.
//
// The two-vector method's dominant step (Section 3.1, Eq. 3; "one lookup per
// group" of Algorithm 1) is a byte load from R at index (h << (q-1)) | c
// followed by an add and a max.  Its analytic ceiling on a Blackwell SM is one
// 32-lane shared-memory wavefront per clock, i.e. 32 lookups/clk/SM when the
// 32 lanes of a warp hit 32 distinct banks.  This microbenchmark measures
// what a full GPU of resident warps actually sustains, in three patterns:
//
//   mode 0, uniform row, indices in registers: every warp-wide lookup reads
//     one row of R (h warp-uniform, a compile-time offset) at the lane's own
//     column c; only the byte load and the max per lookup -- the ceiling of
//     the table-lookup pattern itself;
//   mode 1, uniform row as the fold kernel does it: the row features are
//     packed words (A << 16 | R-row offset) staged in shared memory and read
//     four per 16-byte broadcast load, the lane's column feature (B << 16 | c)
//     sits in a register; per lookup one add, the byte load at the low half,
//     a shift-add of the loaded value into the high half and a max;
//   mode 2, random row: every lane looks up an independent random (h, c), so
//     the warp's 32 bytes fall on random banks (bank conflicts).
//
// Each CTA records its own SM-clock cycles (clock64) around the timed loop;
// the result is lookups per SM-clock per SM with every CTA resident at once
// (grid = SMs x resident CTAs per SM), independent of the clock rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fold.h"

namespace fold {
namespace {

constexpr int kLbThreads = 512;
constexpr int kLbUnroll = 32;

template <int MODE>
__global__ void __launch_bounds__(kLbThreads) lookup_bench_kernel(int q, int iters, long long *cycles,
                                                                 int *sink, int never) {
    extern __shared__ __align__(16) uint8_t lb_smem[];
    const int rbytes = 1 << (2 * (q - 1));
    const int cols = 1 << (q - 1);
    uint8_t *Rs = lb_smem;
    uint32_t *feat = reinterpret_cast<uint32_t *>(lb_smem + rbytes);   // 64 staged row-feature words
    for (int x = threadIdx.x; x < rbytes; x += blockDim.x) Rs[x] = (uint8_t)((x * 2654435761u) >> 29);
    for (int x = threadIdx.x; x < 64; x += blockDim.x)
        feat[x] = ((uint32_t)(x & 7) << 16) | ((uint32_t)((x * 37) & (cols - 1)) << (q - 1));
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    int acc = 0;
    long long t0 = clock64();
    if constexpr (MODE == 0) {
        // the lane's column c; a warp-uniform row offset per outer step; immediate row offsets inside
        const int rows = 1 << (q - 1);
        for (int t = 0; t < iters; ++t) {
            const uint8_t *base = Rs + ((lane + t + warp) & (cols - 1)) + (((t * 7) & (rows - 1) & ~31) << (q - 1));
#pragma unroll
            for (int u = 0; u < kLbUnroll; ++u) acc = max(acc, (int)base[(u & (rows - 1) & 31) << (q - 1)] + u);
        }
    } else if constexpr (MODE == 1) {
        uint32_t cb = ((uint32_t)(lane & 7) << 16) | (uint32_t)(lane & (cols - 1));
        const uint4 *f4 = reinterpret_cast<const uint4 *>(feat);
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int u = 0; u < kLbUnroll / 4; ++u) {
                const uint4 w = f4[(u + t) & 15];
                uint32_t s;
                s = w.x + cb; acc = max(acc, (int)(s + ((uint32_t)Rs[s & 0xffffu] << 16)));
                s = w.y + cb; acc = max(acc, (int)(s + ((uint32_t)Rs[s & 0xffffu] << 16)));
                s = w.z + cb; acc = max(acc, (int)(s + ((uint32_t)Rs[s & 0xffffu] << 16)));
                s = w.w + cb; acc = max(acc, (int)(s + ((uint32_t)Rs[s & 0xffffu] << 16)));
            }
            cb = (cb & 0xffff0000u) | ((cb + 1) & (uint32_t)(cols - 1));
        }
    } else {
        // independent random (h, c) per lane: eight random offsets per lane, each used with four
        // different constant displacements and moved by a warp-uniform amount every step, so the
        // bytes a warp reads at once fall on random banks
        uint32_t off[8];
        uint32_t r = 0x9E3779B9u * (uint32_t)(threadIdx.x + 1) ^ (uint32_t)blockIdx.x * 0x85EBCA6Bu;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            r ^= r << 13; r ^= r >> 17; r ^= r << 5;
            off[u] = r;
        }
        for (int t = 0; t < iters; ++t) {
            const uint32_t shift = (uint32_t)t * 40503u;
#pragma unroll
            for (int u = 0; u < kLbUnroll; ++u)
                acc = max(acc, (int)Rs[(off[u & 7] + shift + (uint32_t)(u >> 3) * 0x2F1A5u) & (uint32_t)(rbytes - 1)] + u);
        }
    }
    long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    if (acc == never) sink[0] = acc;   // `never` is negative at run time: keeps the loop, never stores
}

}  // namespace
}  // namespace fold

using namespace fold;

extern "C" int fold_lookup_rate(int device, int q, int mode, int32_t iters, double *lookups_per_clk_sm,
                                double *kernel_ms) {
    if (q < 2 || q > 9 || mode < 0 || mode > 2 || iters < 1 || iters > (1 << 20) || !lookups_per_clk_sm)
        return FOLD_EINVAL;
    if (mode == 0 && q < 6) return FOLD_EINVAL;   // needs 32 distinct rows and columns
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return FOLD_EINVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) return FOLD_ECUDA;
    const size_t smem = ((size_t)1 << (2 * (q - 1))) + 256;
    void (*kern)(int, int, long long *, int *, int) =
        mode == 0 ? lookup_bench_kernel<0> : (mode == 1 ? lookup_bench_kernel<1> : lookup_bench_kernel<2>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return FOLD_ECUDA;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLbThreads, smem) != cudaSuccess || per_sm < 1)
        return FOLD_ECUDA;
    const int grid = sms * per_sm;
    long long *d_cycles = nullptr;
    int *d_sink = nullptr;
    if (cudaMalloc(&d_cycles, sizeof(long long) * grid) != cudaSuccess) return FOLD_ENOMEM;
    if (cudaMalloc(&d_sink, sizeof(int)) != cudaSuccess) {
        cudaFree(d_cycles);
        return FOLD_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kern<<<grid, kLbThreads, smem>>>(q, iters / 8 + 1, d_cycles, d_sink, -1);   // warm-up
    cudaEventRecord(e0);
    kern<<<grid, kLbThreads, smem>>>(q, iters, d_cycles, d_sink, -1);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long *h = new long long[grid];
    if (e == cudaSuccess) e = cudaMemcpy(h, d_cycles, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    cudaFree(d_cycles);
    cudaFree(d_sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        delete[] h;
        return FOLD_ECUDA;
    }
    long long cmax = 1;
    for (int b = 0; b < grid; ++b) cmax = h[b] > cmax ? h[b] : cmax;
    delete[] h;
    if (cmax < (long long)iters) return FOLD_ECUDA;   // fewer cycles than loop steps: the loop did not run
    const double per_cta = (double)kLbThreads / 32 * 32 * (double)iters * kLbUnroll;   // warps x lanes x lookups
    *lookups_per_clk_sm = per_cta * per_sm / (double)cmax;
    if (kernel_ms) *kernel_ms = ms;
    return FOLD_OK;
}
