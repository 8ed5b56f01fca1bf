// fg.cu -- Section 3.2's FG algorithm (Frid and Gusfield) as a comparison kernel.
//
// FG uses Algorithm 1's groups (group g is full for cell (i,j) iff g*q >= i and g*q+q <= j) and
// residual loops, but instead of one table over all vector pairs it builds a table per row and
// group: when D(i, g*q+q-1) is known, the preprocessing routine runs for row i's own horizontal
// vector h of group g against every vertical vector c and D(i, g*q) is added,
//     FG[i][g][c] = D(i, g*q) + max_{0<=k<=q-1} sum_{p<=k} (h_p - c_p),
// and cell (i,j)'s group term is FG[i][g][c(g,j)] + D(g*q+1, j).  The same horizontal vector is
// tabulated again in every row group where it occurs, which is the duplicated work the paper
// measures.
//
// GPU organisation as in sliding.cu: one warp per column, filled bottom to top; cell (i,j) waits
// (bounded) until column j-1 has done row i, which covers every table FG[i][g] a group reads
// (built by column g*q+q-1 < j at row i); lanes share the cell's groups, residual splits and the
// tabulation of a new row-group table; a warp max-reduction finishes the cell.
//
// Layout (n = sequence length, NG = n/q + 1 groups, NC = 2^(q-1) column vectors): Drow n*n int16
// (zeroed), CV n*NG uint32 with CV[j*NG+g] = (D(g*q+1, j) << 16) | c(g,j), FGT n*NG*NC int16.
#include "fg.h"
#include "fold_kernel.cuh"

namespace fold {

template <int Q>
__global__ void __launch_bounds__(kThreads) fg_kernel(FgParams P) {
    constexpr int NB = Q - 1, NC = 1 << NB;
    constexpr unsigned BM = (1u << NB) - 1;
    const int lane = threadIdx.x & 31;
    const int n = P.n, NG = P.ng;
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(P.next_col, 1);
        j = __shfl_sync(FULL, j, 0);
        if (j >= n) break;
        if (ld_relaxed(P.error) != 0) break;
        const int sj = P.codes[j];
        // win[m] = D(i+m, j) for the cell (i,j) last computed; rows below j count as 0
        int win[Q];
#pragma unroll
        for (int m = 0; m < Q; ++m) win[m] = 0;
        __syncwarp();
        if (lane == 0) st_release(P.progress + j, 1);   // the diagonal cell, D(j,j) = 0
        bool ok = true;
        for (int i = j - 1; i >= 0; --i) {
            const int d = j - i;
            if (!wait_geq_impl(P.progress + (j - 1), d, P.error, P.timeout_ns, lane)) {
                ok = false;
                break;
            }
            const int gfirst = (i + Q - 1) / Q;
            const int glast = j >= Q ? (j - Q) / Q : -1;
            // row i's cells D(i, j-q+1+lane), lane < q-1 (residual splits after the last group and the
            // group a cell at the end of a row group completes)
            const int kc = j - Q + 1 + lane;
            const int rowR = (lane < Q - 1 && kc >= i) ? ldcg16(P.drow + (size_t)i * n + kc) : 0;
            // residual splits, one per lane: k in [i+1, gfirst*q] and [glast*q+q+1, j] when a group is
            // full, else every k in [i+1, j] (at most 2q-2 of them)
            int kr;
            if (gfirst <= glast) {
                const int na = gfirst * Q - i;   // splits before the first group
                kr = lane < na ? i + 1 + lane : glast * Q + Q + 1 + (lane - na);
            } else {
                kr = i + 1 + lane;
            }
            int best = 0;
            if (kr <= j && lane < 2 * Q) {
                // D(i, kr-1) from the columns to the left (L2), D(kr, j) from this warp's own column
                best = ldcg16(P.drow + (size_t)i * n + (kr - 1)) + (kr <= j - 1 ? (int)P.drow[(size_t)kr * n + j] : 0);
            }
            if (lane == 0) {
                const int inner = i + 1 <= j - 1 ? ldcg16(P.drow + (size_t)(i + 1) * n + (j - 1)) : 0;
                best = max(best, inner + (int)((P.pair64 >> (8 * (int)P.codes[i] + sj)) & 1ull));
            }
            // one table read per full group
            for (int g = gfirst + lane; g <= glast; g += 32) {
                const uint32_t cv = P.cv[(size_t)j * NG + g];
                const int t = (int)__ldcg(P.fgt + ((size_t)i * NG + g) * NC + (cv & BM));
                best = max(best, t + (int)(cv >> 16));
            }
            best = __reduce_max_sync(FULL, best);
#pragma unroll
            for (int m = Q - 1; m > 0; --m) win[m] = win[m - 1];
            win[0] = best;
            if (lane == 0) P.drow[(size_t)i * n + j] = (int16_t)best;
            // column j's vector of group g = (i-1)/q is complete once D(g*q+1, j) is known
            if (i >= 1 && (i - 1) % Q == 0 && (i - 1) + Q <= j && lane == 0) {
                unsigned c = 0;
#pragma unroll
                for (int p = 1; p <= NB; ++p) c |= (unsigned)(win[p - 1] - win[p]) << (p - 1);
                P.cv[(size_t)j * NG + (i - 1) / Q] = ((uint32_t)best << 16) | c;
            }
            // row i's group g = (j+1)/q - 1 is complete: tabulate it against every column vector
            if ((j + 1) % Q == 0 && (j + 1) - Q >= i) {
                const int g = (j + 1) / Q - 1;
                const int cur = lane == Q - 1 ? best : rowR;
                const int prev = __shfl_up_sync(FULL, cur, 1);
                const unsigned h = (__ballot_sync(FULL, lane >= 1 && lane <= Q - 1 && cur - prev == 1) >> 1) & BM;
                const int a = __shfl_sync(FULL, rowR, 0);   // D(i, g*q)
                int16_t *row = P.fgt + ((size_t)i * NG + g) * NC;
                for (int c = lane; c < NC; c += 32) {
                    int mv = 0, sum = 0;
#pragma unroll
                    for (int p = 1; p <= NB; ++p) {
                        sum += (int)((h >> (p - 1)) & 1u) - (int)(((unsigned)c >> (p - 1)) & 1u);
                        mv = max(mv, sum);
                    }
                    row[c] = (int16_t)(a + mv);
                }
            }
            if (i == 0 && j == n - 1 && lane == 0) *P.result = best;
            // every lane's stores before lane 0's release (cumulative)
            __syncwarp();
            if (lane == 0) st_release(P.progress + j, d + 1);
        }
        if (!ok) break;
    }
}

template <int Q>
static cudaError_t launch_fg_q(const FgParams &p, int sm_count, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fg_kernel<Q>, kThreads, 0);
    if (e != cudaSuccess) return e;
    const int need = (p.n + kWarpsPerCta - 1) / kWarpsPerCta;
    const int grid = std::max(1, std::min(std::max(per_sm, 1) * sm_count, need));
    fg_kernel<Q><<<grid, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fg(const FgParams &p, int q, int sm_count, cudaStream_t st) {
    switch (q) {
        case 2: return launch_fg_q<2>(p, sm_count, st);
        case 3: return launch_fg_q<3>(p, sm_count, st);
        case 4: return launch_fg_q<4>(p, sm_count, st);
        case 5: return launch_fg_q<5>(p, sm_count, st);
        case 6: return launch_fg_q<6>(p, sm_count, st);
        case 7: return launch_fg_q<7>(p, sm_count, st);
        case 8: return launch_fg_q<8>(p, sm_count, st);
        case 9: return launch_fg_q<9>(p, sm_count, st);
        case 10: return launch_fg_q<10>(p, sm_count, st);
    }
    return cudaErrorInvalidValue;
}

FgLayout fg_layout(int n, int q) {
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    FgLayout L;
    const size_t nn = (size_t)std::max(n, 1);
    L.ng = (int)(nn / (size_t)q + 1);
    L.off_control = 0;
    L.off_results = 256;
    L.off_progress = 512;
    L.zero_bytes = al(L.off_progress + 4 * nn);
    L.off_codes = L.zero_bytes;
    L.off_drow = al(L.off_codes + nn);
    L.off_cv = al(L.off_drow + 2 * nn * nn);
    L.off_fgt = al(L.off_cv + 4 * nn * (size_t)L.ng);
    L.bytes = al(L.off_fgt + 2 * nn * (size_t)L.ng * ((size_t)1 << (q - 1)));
    return L;
}

}  // namespace fold
