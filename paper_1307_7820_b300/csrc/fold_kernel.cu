// fold_kernel.cu -- small kernels of libfold_b300 and the dispatch to the
// per-instantiation launchers (fold_inst_*.cu).
//
//   rtable_build_kernel   Section 3.1 preprocessing: one thread per pair of
//                         (q-1)-bit difference vectors.
//   extract / pad / finalize   data movement around the persistent kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fold_common.h"
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
// D(i,k-1) + D(k,j).  One block: thread 0 follows unpaired bases and pairs (each step reads two
// cells), the whole block searches a split's k range, blockDim candidates at a time.  The pending
// intervals live in `stack` (n entries).  partner[x] = the base paired with x, or -1.  *result is
// the fold's answer D(0,n-1) (or -status if the fold failed, then nothing is traced); it becomes
// -fail_code if the trace finds no argmax somewhere, runs past its step bound, or ends with a
// different number of pairs (the table would not be one of Eq. 1).
__global__ void traceback_kernel(const int16_t *Drow, int Np, const uint8_t *codes, int n, unsigned long long pair64,
                                 int2 *stack, int32_t *partner, int32_t *result, int fail_code) {
    __shared__ int s_i, s_j, s_dij, s_k, s_act;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int x = tid; x < n; x += nt) partner[x] = -1;
    // the fold failed (its answer is -status): no table to trace
    if (*(volatile const int32_t *)result < 0) return;
    int status = 0, pairs = 0;   // thread 0's
    auto DV = [&](int a, int b) -> int { return a >= b ? 0 : (int)Drow[(size_t)a * Np + b]; };
    int top = 0, steps = 0;   // thread 0's stack depth and step count
    int ci = 0, cj = n - 1;   // thread 0's current interval (empty when ci >= cj)
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            int act = 0;   // 0: finished, 2: a split to search
            for (;;) {
                if (ci >= cj) {
                    if (top == 0) break;
                    const int2 e = stack[--top];
                    ci = e.x;
                    cj = e.y;
                    continue;
                }
                if (++steps > 4 * n + 8) {
                    status = 1;
                    break;
                }
                const int dij = DV(ci, cj);
                if (dij == DV(ci + 1, cj)) {   // base ci unpaired
                    ++ci;
                    continue;
                }
                if (((pair64 >> (8 * codes[ci] + codes[cj])) & 1ull) && dij == DV(ci + 1, cj - 1) + 1) {
                    partner[ci] = cj;
                    partner[cj] = ci;
                    ++pairs;
                    ++ci;
                    --cj;
                    continue;
                }
                s_i = ci;
                s_j = cj;
                s_dij = dij;
                s_k = 0x7fffffff;
                act = 2;
                break;
            }
            s_act = act;
        }
        __syncthreads();
        if (s_act == 0) break;
        const int i = s_i, j = s_j, dij = s_dij;
        for (int base = i + 2; base <= j; base += nt) {
            const int k = base + tid;
            if (k <= j && DV(i, k - 1) + DV(k, j) == dij) atomicMin(&s_k, k);
            __syncthreads();
            const bool found = s_k != 0x7fffffff;
            __syncthreads();
            if (found) break;
        }
        if (tid == 0) {
            const int k = s_k;
            if (k == 0x7fffffff || top >= n) {   // no argmax: stop
                status = 2;
                ci = cj = 0;
                top = 0;
            } else {
                stack[top++] = make_int2(k, j);
                ci = i;
                cj = k - 1;
            }
        }
        __syncthreads();
    }
    // a structure with as many pairs as the answer, or the answer becomes -fail_code
    if (tid == 0 && (status != 0 || pairs != *result)) *result = -fail_code;
}

cudaError_t launch_traceback(const int16_t *drow, int Np, const uint8_t *codes, int n, unsigned long long pair64,
                             int2 *stack, int32_t *partner, int32_t *result, int fail_code, cudaStream_t st) {
    traceback_kernel<<<1, 256, 0, st>>>(drow, Np, codes, n, pair64, stack, partner, result, fail_code);
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

cudaError_t launch_pad_codes(const uint8_t *in, int n, int Np, uint8_t *out, cudaStream_t st) {
    int blocks = (Np + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    pad_codes_kernel<<<blocks, 256, 0, st>>>(in, n, Np, out);
    return cudaGetLastError();
}

}  // namespace fold
