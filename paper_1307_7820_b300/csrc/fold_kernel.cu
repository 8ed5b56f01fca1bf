// fold_kernel.cu -- small kernels of libfold_b300 and the dispatch to the
// per-instantiation launchers (fold_inst_*.cu).
//
//   rtable_build_kernel   Section 3.1 preprocessing: one thread per pair of
//                         (q-1)-bit difference vectors.
//   extract / pad / finalize   data movement around the persistent kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <stdint.h>

#include "fold_common.h"
#include "fold_kernel.cuh"
#include "kernels.h"

namespace fold {

#define FOLD_INST_DECL(NAME) \
    cudaError_t launch_##NAME(const FoldParams &p, int grid, cudaStream_t st); \
    int bps_##NAME(); \
    size_t smem_##NAME();
FOLD_INST_DECL(tv2)
FOLD_INST_DECL(tv3)
FOLD_INST_DECL(tv4)
FOLD_INST_DECL(tv5)
FOLD_INST_DECL(tv6)
FOLD_INST_DECL(tv7)
FOLD_INST_DECL(tv8)
FOLD_INST_DECL(tv9)
FOLD_INST_DECL(tv10)
FOLD_INST_DECL(plain)
cudaError_t launch_memo2(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo3(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo4(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo5(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo6(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo7(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo8(const FoldParams &p, int grid, cudaStream_t st);
cudaError_t launch_memo9(const FoldParams &p, int grid, cudaStream_t st);

// ------------------------------------------------------------------ R table
// R[(h << (q-1)) | c] = max over k in [0,q-1] of sum_{p<=k} (h_p - c_p), with
// h_0 = c_0 = 0 (the scan of the preprocessing routine, strict '>' from 0).
__global__ void rtable_build_kernel(int q, uint8_t *canon, uint8_t *packed) {
    int nb = q - 1;
    long long nent = 1LL << (2 * nb);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nent;
         idx += (long long)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)(idx >> nb), c = (unsigned)(idx & ((1u << nb) - 1));
        int best = 0, sum = 0;
        for (int p = 1; p <= nb; ++p) {
            sum += (int)((h >> (p - 1)) & 1u) - (int)((c >> (p - 1)) & 1u);
            if (sum > best) best = sum;
        }
        canon[idx] = (uint8_t)best;
    }
    // packed form used by the kernel: bytes for q <= 9, nibbles for q = 10
    if (q >= 10) {
        for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nent / 2;
             b += (long long)gridDim.x * blockDim.x) {
            unsigned h = (unsigned)((2 * b) >> nb), c0 = (unsigned)((2 * b) & ((1u << nb) - 1));
            int v[2];
            for (int e = 0; e < 2; ++e) {
                unsigned c = c0 + e;
                int best = 0, sum = 0;
                for (int p = 1; p <= nb; ++p) {
                    sum += (int)((h >> (p - 1)) & 1u) - (int)((c >> (p - 1)) & 1u);
                    if (sum > best) best = sum;
                }
                v[e] = best;
            }
            packed[b] = (uint8_t)(v[0] | (v[1] << 4));
        }
    }
}

// ---------------------------------------------------------------- extract
// Dense n*n row-major copy of the upper triangle (0 below the diagonal).
__global__ void extract_kernel(const int16_t *drow, int Np, int n, int16_t *out) {
    long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / n), jj = (int)(e % n);
        out[e] = (i <= jj) ? drow[(size_t)i * Np + jj] : (int16_t)0;
    }
}

// Pads 2-bit codes to Np with the padding code.
__global__ void pad_codes_kernel(const uint8_t *in, int n, int Np, uint8_t *out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Np; e += gridDim.x * blockDim.x)
        out[e] = (e < n) ? in[e] : (uint8_t)kPadCode;
}

// ---------------------------------------------------------------- host side
size_t fold_smem_bytes(int q, int method) {
    if (method == kPlain) return smem_plain();
    switch (q) {
        case 2: return smem_tv2();
        case 3: return smem_tv3();
        case 4: return smem_tv4();
        case 5: return smem_tv5();
        case 6: return smem_tv6();
        case 7: return smem_tv7();
        case 8: return smem_tv8();
        case 9: return smem_tv9();
        case 10: return smem_tv10();
    }
    return 0;
}

bool fold_col_helpers_supported(int q, int method) {
    if (method != kTwoVector) return false;
    switch (q) {
        case 2: return col_helpers_fit<2>();
        case 3: return col_helpers_fit<3>();
        case 4: return col_helpers_fit<4>();
        case 5: return col_helpers_fit<5>();
        case 6: return col_helpers_fit<6>();
        case 7: return col_helpers_fit<7>();
        case 8: return col_helpers_fit<8>();
        case 9: return col_helpers_fit<9>();
        case 10: return col_helpers_fit<10>();
    }
    return false;
}

int fold_blocks_per_sm(int q, int method) {
    if (method == kPlain) return bps_plain();
    switch (q) {
        case 2: return bps_tv2();
        case 3: return bps_tv3();
        case 4: return bps_tv4();
        case 5: return bps_tv5();
        case 6: return bps_tv6();
        case 7: return bps_tv7();
        case 8: return bps_tv8();
        case 9: return bps_tv9();
        case 10: return bps_tv10();
    }
    return 0;
}

// ------------------------------------------------------------------ traceback
// Section 2: one optimal structure from a finished table.  The paper keeps D* (the argmax of Eq. 1)
// beside D; here the argmax is re-evaluated from D at each cell visited, in a fixed order of
// preference: the split k = i+1 (base i unpaired) if D(i,j) = D(i+1,j); else the pair (i,j) if
// b(S_i,S_j) = 1 and D(i,j) = D(i+1,j-1) + 1; else the smallest k in [i+2, j] with D(i,j) =
// D(i,k-1) + D(k,j).  The two intervals a split leaves, [i, k-1] and [k, j], are traced
// independently, so warps take intervals from a queue: a warp walks its interval and, at a split,
// queues [k, j] and goes on with [i, k-1].  The result does not depend on which warp traces what.
// Walking: an 8 x 16 window of the table (rows i+1.., columns ..j) and the bases of its rows and
// columns are staged in shared memory by one round of loads and serve the unpaired and pair steps
// inside it; a split's k range is searched 128 candidates per round (4 per lane, ballots in
// increasing k).  Queue: slots claimed in order (head) and published with a release of
// ready[slot]; one 64-bit word counts queued intervals (high half, which also numbers the slots)
// and finished ones (low half): the trace is over when they are equal, so a warp waiting on a slot
// that is never filled stops then.  Every wait is bounded.  partner[x] = the base paired with x, or
// -1 (set by the caller).
namespace {
constexpr int kTbLine = 32;                  // ints per 128-byte line: each counter on its own line
constexpr int kTbRows = 8, kTbCols = 16;     // window of the walk
constexpr int kTbWarps = 4;                  // warps per block
struct TbArgs {
    const int16_t *Drow;
    int Np, n;
    const uint8_t *codes;
    unsigned long long pair64;
    int2 *queue;       // intervals (n + 2 slots)
    int *qval;         // D of each queued interval
    int *ready;        // slot published (zeroed by the caller)
    int *state;        // head | queued-finished word | pairs | error, kTbLine ints apart
    int32_t *partner;
    const int32_t *result;
    long long timeout_ns;
};
}

__global__ void traceback_init_kernel(TbArgs A) {
    // the fold failed (its answer is -status): nothing to trace
    const int root = *(volatile const int32_t *)A.result;
    A.state[0] = 0;
    *reinterpret_cast<unsigned long long *>(A.state + kTbLine) = root >= 0 ? (1ull << 32) : 0ull;
    A.state[2 * kTbLine] = 0;
    A.state[3 * kTbLine] = 0;
    if (root >= 0) {
        A.queue[0] = make_int2(0, A.n - 1);
        A.qval[0] = root;
        A.ready[0] = 1;
    }
}

static __device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(32 * kTbWarps) traceback_par_kernel(TbArgs A) {
    __shared__ int16_t s_win[kTbWarps][kTbRows][kTbCols];
    __shared__ uint8_t s_br[kTbWarps][kTbRows], s_bc[kTbWarps][kTbCols];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    int *head = A.state, *err = A.state + 3 * kTbLine;
    unsigned long long *qf = reinterpret_cast<unsigned long long *>(A.state + kTbLine);
    const int cap = A.n + 2, n = A.n, Np = A.Np;
    auto DV = [&](int a, int b) -> int { return a >= b ? 0 : (int)__ldcg(A.Drow + (size_t)a * Np + b); };
    int pairs = 0;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(head, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= cap) break;
        int ok = 0;
        if (lane == 0) {
            const unsigned long long t0 = gtimer();
            unsigned ns = 32;
            for (unsigned it = 0;; ++it) {
                if (ld_acquire(A.ready + idx)) { ok = 1; break; }
                if ((it & 7u) == 7u) {   // the shared counters, seldom
                    const unsigned long long v = ld_acquire64(qf);
                    if ((unsigned)(v >> 32) == (unsigned)v || ld_relaxed(err) != 0) break;
                    if ((long long)(gtimer() - t0) > A.timeout_ns) {
                        atomicCAS(err, 0, 1);
                        break;
                    }
                }
                __nanosleep(ns);
                ns = ns < 256 ? 2 * ns : 256;
            }
        }
        if (!__shfl_sync(FULL, ok, 0)) break;
        const int2 e = __ldcg(A.queue + idx);
        int i = e.x, j = e.y, dij = __ldcg(A.qval + idx);
        bool bad = false;
        while (i < j && !bad) {
            // window: rows i+1..i+8, columns j-15..j (4 cells per lane), and its bases
            const int wi = i, wj = j;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int cell = lane * 4 + u;
                const int r = wi + 1 + cell / kTbCols, cc = wj - (kTbCols - 1) + cell % kTbCols;
                s_win[wp][cell / kTbCols][cell % kTbCols] = (int16_t)((cc >= 0 && r < n) ? DV(r, cc) : 0);
            }
            if (lane < kTbRows) s_br[wp][lane] = wi + lane < n ? A.codes[wi + lane] : 0;
            if (lane < kTbCols) s_bc[wp][lane] = wj - lane >= 0 ? A.codes[wj - lane] : 0;
            __syncwarp();
            bool split = false;
            for (;;) {
                if (i >= j) break;
                const int dr = i - wi, dc = j - (wj - (kTbCols - 1));   // row i+1 of the window, column j
                if (dr > kTbRows - 1 || dc < 1) break;                   // left the window: load the next one
                if (dij == (int)s_win[wp][dr][dc]) {                     // base i unpaired
                    ++i;
                    continue;
                }
                const int bi = s_br[wp][dr], bj = s_bc[wp][wj - j];
                if (((A.pair64 >> (8 * bi + bj)) & 1ull) && dij == (int)s_win[wp][dr][dc - 1] + 1) {
                    if (lane == 0) {
                        A.partner[i] = j;
                        A.partner[j] = i;
                    }
                    ++pairs;
                    ++i;
                    --j;
                    --dij;
                    continue;
                }
                split = true;
                break;
            }
            if (i >= j || !split) continue;
            // the smallest split k in [i+2, j]: 128 candidates in the first round (most splits are
            // near i), then 1024 a round, all of a round's loads in flight at once
            int k = -1, dl = 0, dk = 0;
            auto scan = [&](auto width_tag, int base) {
                constexpr int U = decltype(width_tag)::value;
                int a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int kk = base + 32 * u + lane;
                    a[u] = kk <= j ? DV(i, kk - 1) : 0;
                    b[u] = kk <= j ? DV(kk, j) : 0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int kk = base + 32 * u + lane;
                    const unsigned m = __ballot_sync(FULL, kk <= j && a[u] + b[u] == dij);
                    if (m && k < 0) {
                        const int src = __ffs(m) - 1;
                        k = base + 32 * u + src;
                        dl = __shfl_sync(FULL, a[u], src);
                        dk = __shfl_sync(FULL, b[u], src);
                    }
                }
            };
            scan(std::integral_constant<int, 4>(), i + 2);
            for (int base = i + 2 + 128; base <= j && k < 0; base += 1024) scan(std::integral_constant<int, 32>(), base);
            if (k < 0) {   // no argmax: the table is not one of Eq. 1
                bad = true;
                if (lane == 0) atomicCAS(err, 0, 2);
                break;
            }
            if (lane == 0) {
                const int slot = (int)(atomicAdd(qf, 1ull << 32) >> 32);
                if (slot < cap) {
                    A.queue[slot] = make_int2(k, j);
                    A.qval[slot] = dk;
                    st_release(A.ready + slot, 1);
                } else {
                    atomicCAS(err, 0, 3);
                }
            }
            j = k - 1;
            dij = dl;
        }
        __syncwarp();
        if (lane == 0) atomicAdd(qf, 1ull);   // this interval is finished
        if (bad) break;
    }
    if (lane == 0 && pairs) atomicAdd(A.state + 2 * kTbLine, pairs);
}

__global__ void traceback_check_kernel(TbArgs A, int fail_code) {
    const int root = *A.result;
    if (root < 0) return;
    if (A.state[3 * kTbLine] != 0 || A.state[2 * kTbLine] != root) *const_cast<int32_t *>(A.result) = -fail_code;
}

size_t traceback_scratch_bytes(int n) {
    const size_t cap = (size_t)std::max(n, 1) + 2;
    return ((8 * cap + 255) / 256 + (4 * cap + 255) / 256 + (4 * cap + 255) / 256) * 256 + 4 * kTbLine * 4;
}

cudaError_t launch_traceback(const int16_t *drow, int Np, const uint8_t *codes, int n, unsigned long long pair64,
                             void *scratch, int32_t *partner, int32_t *result, int fail_code, long long timeout_ns,
                             int sm_count, cudaStream_t st) {
    const size_t cap = (size_t)std::max(n, 1) + 2;
    uint8_t *b = reinterpret_cast<uint8_t *>(scratch);
    TbArgs A;
    A.Drow = drow;
    A.Np = Np;
    A.n = n;
    A.codes = codes;
    A.pair64 = pair64;
    A.queue = reinterpret_cast<int2 *>(b);
    A.qval = reinterpret_cast<int *>(b + (8 * cap + 255) / 256 * 256);
    A.ready = reinterpret_cast<int *>(b + ((8 * cap + 255) / 256 + (4 * cap + 255) / 256) * 256);
    A.state = reinterpret_cast<int *>(b + ((8 * cap + 255) / 256 + 2 * ((4 * cap + 255) / 256)) * 256);
    A.partner = partner;
    A.result = result;
    A.timeout_ns = timeout_ns;
    cudaError_t e = cudaMemsetAsync(A.ready, 0, 4 * cap, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(partner, 0xff, 4 * (size_t)n, st);
    if (e != cudaSuccess) return e;
    traceback_init_kernel<<<1, 1, 0, st>>>(A);
    // enough warps for the intervals open at once (a few hundred at most for long folds)
    const int blocks = std::max(1, std::min(sm_count, (n + 255) / 256));
    traceback_par_kernel<<<blocks, 32 * kTbWarps, 0, st>>>(A);
    traceback_check_kernel<<<1, 1, 0, st>>>(A, fail_code);
    return cudaGetLastError();
}

// Writes the answers (or -status if any device-side wait failed).
__global__ void finalize_kernel(const int *error, const int *results, int count, int32_t *out) {
    int e = *(volatile const int *)error;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x)
        out[k] = e == kErrNone ? results[k] : (e == kErrTimeout ? -4 : -1);
}

cudaError_t launch_finalize(const int *error, const int *results, int count, int32_t *out, cudaStream_t st) {
    int blocks = (count + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    finalize_kernel<<<blocks, 256, 0, st>>>(error, results, count, out);
    return cudaGetLastError();
}

cudaError_t launch_fold(const FoldParams &p, int q, int method, int grid, cudaStream_t st) {
    if (method == kPlain) return launch_plain(p, grid, st);
    if (p.memo) {   // Section 3.2's partially memoised table (same shared memory and occupancy)
        switch (q) {
            case 2: return launch_memo2(p, grid, st);
            case 3: return launch_memo3(p, grid, st);
            case 4: return launch_memo4(p, grid, st);
            case 5: return launch_memo5(p, grid, st);
            case 6: return launch_memo6(p, grid, st);
            case 7: return launch_memo7(p, grid, st);
            case 8: return launch_memo8(p, grid, st);
            case 9: return launch_memo9(p, grid, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (q) {
        case 2: return launch_tv2(p, grid, st);
        case 3: return launch_tv3(p, grid, st);
        case 4: return launch_tv4(p, grid, st);
        case 5: return launch_tv5(p, grid, st);
        case 6: return launch_tv6(p, grid, st);
        case 7: return launch_tv7(p, grid, st);
        case 8: return launch_tv8(p, grid, st);
        case 9: return launch_tv9(p, grid, st);
        case 10: return launch_tv10(p, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rtable(int q, uint8_t *canon, uint8_t *packed, cudaStream_t st) {
    long long nent = 1LL << (2 * (q - 1));
    int blocks = (int)((nent + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    rtable_build_kernel<<<blocks, 256, 0, st>>>(q, canon, packed);
    return cudaGetLastError();
}

cudaError_t launch_extract(const int16_t *drow, int Np, int n, int16_t *out, cudaStream_t st) {
    long long total = (long long)n * n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    extract_kernel<<<blocks, 256, 0, st>>>(drow, Np, n, out);
    return cudaGetLastError();
}

// A batch's task list from device copies of the per-size templates: segment s = {first task in the
// store, count, sequence index, position in the list}; a warp copies one segment, rewriting the
// sequence index of every task.
__global__ void gather_tasks_kernel(const int4 *__restrict__ store, const int4 *__restrict__ segs, int nseg,
                                    int4 *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += warps) {
        const int4 sg = __ldg(segs + s);
        for (int e = lane; e < sg.y; e += 32) {
            int4 v = __ldg(store + (size_t)sg.x + e);
            v.x = sg.z;
            out[(size_t)sg.w + e] = v;
        }
    }
}

cudaError_t launch_gather_tasks(const int4 *store, const int4 *segs, int nseg, int4 *out, int sm_count,
                                cudaStream_t st) {
    if (nseg <= 0) return cudaSuccess;
    const int blocks = std::max(1, std::min((nseg + 7) / 8, 8 * std::max(sm_count, 1)));
    gather_tasks_kernel<<<blocks, 256, 0, st>>>(store, segs, nseg, out);
    return cudaGetLastError();
}

cudaError_t launch_pad_codes(const uint8_t *in, int n, int Np, uint8_t *out, cudaStream_t st) {
    int blocks = (Np + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    pad_codes_kernel<<<blocks, 256, 0, st>>>(in, n, Np, out);
    return cudaGetLastError();
}

}  // namespace fold
