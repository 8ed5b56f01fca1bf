// sliding.cu -- Section 4's parallel two-vector algorithm with difference vectors at every cell
// (the sliding-window variant), kept as a second kernel organisation beside the tiled kernel.
//
// Section 4 gives every column j a process that fills the column bottom to top, all processes
// advancing one diagonal per iteration.  Per cell (i,j): the pair term D(i+1,j-1) + b(S_i,S_j);
// one table lookup per group of q splits starting at i, D(i,k) + D(k+1,j) + R[dH(i,k)][dV(k+1,j)]
// for k = i + k'q, k' < floor((j-i)/q); the residual splits k = i + floor((j-i)/q)q .. j-1; then the
// two vectors the cell completes are stored, dV(i,j) (cells D(i..i+q-1, j)) and dH(i, j-q+1) (cells
// D(i, j-q+1..j)).  Vectors are kept for every cell so that every process does the same work.
//
// Here a process is a warp: its lanes share a cell's lookups (lane l takes k' = l, l+32, ...) and
// a warp max-reduction finishes the cell.  Instead of a barrier per diagonal, column j publishes
// how many of its rows are done; cell (i,j) waits (bounded) until column j-1 has done row i, which
// by induction covers everything the cell reads: D(i+1,j-1), row i left of j, and every horizontal
// vector of row i that a group reads.  Warps take columns in increasing order from one counter, so
// the lowest unfinished column never waits on an unfinished one and the fold needs no
// co-residency.
//
// Layout (n = sequence length, no padding): Drow n*n int16 row-major (zeroed: cells below the
// diagonal are 0), H n*n uint32 row-major with H[i*n+k] = (D(i,k) << 16) | R-row offset of dH(i,k)
// (dH itself for nibble tables), V n*n uint32 column-major with V[j*n+r] = (D(r,j) << 16) | dV(r,j);
// the words are group_term's operands.
#include "fold_kernel.cuh"
#include "sliding.h"

namespace fold {

template <int Q>
__global__ void __launch_bounds__(kThreads) sliding_kernel(SlidingParams P) {
    using C = Cfg<Q, kTwoVector>;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *Rs = smem;
    if constexpr (C::RBYTES > 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.rtab);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (int v = threadIdx.x; v < (C::RBYTES + 15) / 16; v += blockDim.x) dst[v] = __ldg(src + v);
    }
    // per warp: the bottom cells of the current column, cb[m] = D(j-m, j) for m < q
    int *cb = reinterpret_cast<int *>(smem + round_up(C::RBYTES, 128)) + warp * 16;
    __syncthreads();
    const int n = P.n;
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(P.next_col, 1);
        j = __shfl_sync(FULL, j, 0);
        if (j >= n) break;
        if (ld_relaxed(P.error) != 0) break;
        const int sj = P.codes[j];
        uint32_t *Vcol = P.V + (size_t)j * n;
        // win[m] = D(i+m, j) for the cell (i,j) last computed; rows below j count as 0
        int win[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) win[m] = 0;
        // the diagonal cell: D(j,j) = 0 (the table is zeroed), dV(j,j) = (0, 0)
        if (lane == 0) {
            cb[0] = 0;
            Vcol[j] = 0u;
        }
        __syncwarp();
        if (lane == 0) st_release(P.progress + j, 1);
        bool ok = true;
        for (int i = j - 1; i >= 0; --i) {
            const int d = j - i;
            // column j-1 has done row i (d rows counted from its diagonal)
            if (!wait_geq_impl(P.progress + (j - 1), d, P.error, P.timeout_ns, lane)) {
                ok = false;
                break;
            }
            const int G = d / Q;
            const int k0 = j - Q + 1;
            // row i's cells D(i, k0+lane) for lane < q-1 (the residual splits' left parts and dH(i,k0))
            const int kc = k0 + lane;
            const int rowv = (lane < Q - 1 && kc >= i) ? ldcg16(P.drow + (size_t)i * n + kc) : 0;
            const int inner = (lane == 0 && i + 1 <= j - 1) ? ldcg16(P.drow + (size_t)(i + 1) * n + (j - 1)) : 0;
            // groups relative to i: k = i + k'q, one lookup each
            int gbest = (int)0x80000000u;
            const uint32_t *Hrow = P.H + (size_t)i * n;
#pragma unroll 4
            for (int kp = lane; kp < G; kp += 32) {
                const int k = i + kp * Q;
                gbest = max(gbest, group_term<Q>(Rs, __ldcg(Hrow + k), Vcol[k + 1]));
            }
            // residual splits k = i + G*q + lane <= j-1: D(i,k) + D(k+1,j), D(k+1,j) = cb[j-k-1]
            const int kr = i + G * Q + lane;
            const int dik = __shfl_sync(FULL, rowv, (kr - k0) & 31);
            int best = (lane < Q - 1 && kr <= j - 1) ? dik + cb[min(max(j - kr - 1, 0), 15)] : 0;
            if (lane == 0) best = max(best, inner + (int)((P.pair64 >> (8 * (int)P.codes[i] + sj)) & 1ull));
            best = max(best, gbest >> 16);
            best = __reduce_max_sync(FULL, best);
            // the cell and the vectors it completes
#pragma unroll
            for (int m = Q - 1; m > 0; --m) win[m] = win[m - 1];
            win[0] = best;
            unsigned bv = 0;
#pragma unroll
            for (int p = 1; p < Q; ++p) bv |= (unsigned)(win[p - 1] - win[p]) << (p - 1);
            uint32_t hword = 0;
            if (k0 >= i) {
                // dH(i,k0): bit p-1 = D(i,k0+p) - D(i,k0+p-1), the cells in lanes 0..q-2 and D(i,j)
                const int cur = lane == Q - 1 ? best : rowv;
                const int prev = __shfl_up_sync(FULL, cur, 1);
                const unsigned hb = __ballot_sync(FULL, lane >= 1 && lane <= Q - 1 && cur - prev == 1);
                const unsigned bits = (hb >> 1) & C::BMASK;
                const int a = __shfl_sync(FULL, rowv, 0);
                hword = ((uint32_t)a << 16) | (C::NIB ? bits : (uint32_t)hrow_offset<Q>((int)bits));
            }
            if (lane == 0) {
                P.drow[(size_t)i * n + j] = (int16_t)best;
                Vcol[i] = ((uint32_t)best << 16) | bv;
                if (k0 >= i) P.H[(size_t)i * n + k0] = hword;
                if (d < Q) cb[d] = best;
                if (i == 0 && j == n - 1) *P.result = best;
            }
            __syncwarp();
            // lane 0 made every store above; its release publishes them with the count
            if (lane == 0) st_release(P.progress + j, d + 1);
        }
        if (!ok) break;
    }
}

template <int Q>
static cudaError_t launch_sliding_q(const SlidingParams &p, int sm_count, cudaStream_t st) {
    const size_t smem = (size_t)round_up(Cfg<Q, kTwoVector>::RBYTES, 128) + (size_t)kWarpsPerCta * 16 * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(sliding_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sliding_kernel<Q>, kThreads, smem);
    if (e != cudaSuccess) return e;
    // persistent: as many warps as fit, never more than one per column
    const int need = (p.n + kWarpsPerCta - 1) / kWarpsPerCta;
    const int grid = std::max(1, std::min(std::max(per_sm, 1) * sm_count, need));
    sliding_kernel<Q><<<grid, kThreads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sliding(const SlidingParams &p, int q, int sm_count, cudaStream_t st) {
    switch (q) {
        case 2: return launch_sliding_q<2>(p, sm_count, st);
        case 3: return launch_sliding_q<3>(p, sm_count, st);
        case 4: return launch_sliding_q<4>(p, sm_count, st);
        case 5: return launch_sliding_q<5>(p, sm_count, st);
        case 6: return launch_sliding_q<6>(p, sm_count, st);
        case 7: return launch_sliding_q<7>(p, sm_count, st);
        case 8: return launch_sliding_q<8>(p, sm_count, st);
        case 9: return launch_sliding_q<9>(p, sm_count, st);
        case 10: return launch_sliding_q<10>(p, sm_count, st);
    }
    return cudaErrorInvalidValue;
}

SlidingLayout sliding_layout(int n) {
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    SlidingLayout L;
    const size_t nn = (size_t)std::max(n, 1);
    L.off_control = 0;                                    // next column, error word
    L.off_results = 256;
    L.off_progress = 512;
    L.zero_bytes = al(L.off_progress + 4 * nn);
    L.off_codes = L.zero_bytes;
    L.off_drow = al(L.off_codes + nn);
    L.off_H = al(L.off_drow + 2 * nn * nn);
    L.off_V = al(L.off_H + 4 * nn * nn);
    L.bytes = al(L.off_V + 4 * nn * nn);
    return L;
}

}  // namespace fold
