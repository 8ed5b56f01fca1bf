// fold_kernel.cuh -- device code of the persistent fold kernel (sm_103a).
// Included by one fold_inst_*.cu file per instantiation.
//
//   fold_kernel<Q,M>      persistent dataflow kernel: every warp is a worker
//                         that takes tasks (NEAR tile / FAR chunk, see
//                         schedule.cpp) from one ordered list.  M selects the
//                         two-vector method (group lookups in R, Eq. 3) or the
//                         plain Nussinov recurrence (Eq. 1) kept as the
//                         comparison; both share the schedule and the tile
//                         recurrence, so they differ only in the split loops.
//
// Tile recurrence (NEAR).  Inside tile (I,J) rows are processed bottom-up.
// For row i, Y_c collects everything that does not read row i itself: the
// pair term b(S_i,S_j) + D(i+1,j-1), the far partial max P, and the splits
// whose right part D(k,j) lies in the current tile column below row i.  The
// splits whose left part D(i,k-1) lies in the current row are then folded in
// by the closure D_c = max(Y_c, max_{c'<c} Y_c' + W[c'][c]), W[c'][c] =
// D(JT+c'+1, JT+c) from diagonal tile (J,J).  This is exact: unrolling the
// in-row dependency gives paths c_0 < ... < c, and superadditivity of D
// (Eq. 1 with split k) makes every path of length >= 2 no better than a
// direct one.  It turns the in-row chain into one data-parallel step.
//
// Difference vectors (Section 3.1).  When the tile's row i is final, its
// horizontal vectors are packed with one warp ballot (bit c = D(i,JT+c) -
// D(i,JT+c-1)); each lane keeps the vertical differences of its column in a
// shift register.  Features are stored packed as (base << 16) | bits.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fold_common.h"

namespace fold {

#ifndef FULL
#define FULL 0xffffffffu
#endif

// ------------------------------------------------------------------ helpers
static __device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Lane 0 waits (bounded) until *p >= target; the verdict is broadcast.  On
// timeout the error word is set; any error seen makes every worker stop.
static __device__ __noinline__ bool wait_geq_impl(const int *p, int target, int *error, long long timeout_ns, int lane) {
    int ok = 1;
    if (lane == 0) {
        if (ld_acquire(p) < target) {
            unsigned long long t0 = gtimer();
            unsigned ns = 64;
            for (;;) {
                __nanosleep(ns);
                if (ns < 2048) ns <<= 1;
                if (ld_acquire(p) >= target) break;
                if (*(volatile int *)error != 0) { ok = 0; break; }
                if ((long long)(gtimer() - t0) > timeout_ns) {
                    atomicCAS(error, 0, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        }
    }
    ok = __shfl_sync(FULL, ok, 0);
    __syncwarp();
    return ok != 0;
}
static __device__ __forceinline__ bool warp_wait_geq(const int *p, int target, const FoldParams &P, int lane) {
    return wait_geq_impl(p, target, P.error, P.timeout_ns, lane);
}

static __device__ __forceinline__ int lds16(const int16_t *p) { return (int)*p; }
static __device__ __forceinline__ int ldcg16(const int16_t *p) { return (int)__ldcg(p); }

template <int Q, int M>
struct Cfg {
    static constexpr int T = tile_of(Q, M);
    static constexpr int G = (M == kPlain) ? 1 : T / Q;   // groups per tile edge
    static constexpr int NB = Q - 1;                          // free bits per vector
    static constexpr unsigned BMASK = (1u << NB) - 1;
    static constexpr bool NIB = (M == kTwoVector) && (Q >= 10);
    static constexpr int RBYTES = (M == kPlain) ? 0 : (NIB ? (1 << (2 * NB - 1)) : (1 << (2 * NB)));
};

// per-warp shared scratch
template <int Q, int M>
struct __align__(16) WarpScratch {
    static constexpr int T = Cfg<Q, M>::T;
    static constexpr int G = Cfg<Q, M>::G;
    int2 rf[G][32];                 // far staging (two-vector): (A, h-row byte offset)
    alignas(16) int16_t rows[32][32];  // far staging (plain): row strips (uint4 access)
    int16_t diag[T][T + 2];         // diagonal tile (I,I) rows
    uint32_t drf[T][G];             // diagonal tile row features
    alignas(16) int16_t y[32];      // closure exchange (read back as uint4)
    int16_t left[T + 2];            // D(IT+m, JT-1)
    int16_t tile[T][T + 1];         // output tile (transposed store)
};

// every vector-accessed member must sit on a 16-byte boundary
template <int Q, int M>
struct ScratchChecks {
    using WS = WarpScratch<Q, M>;
    static_assert(offsetof(WS, y) % 16 == 0, "y must be 16-byte aligned");
    static_assert(offsetof(WS, rows) % 16 == 0, "rows must be 16-byte aligned");
    static_assert(sizeof(WarpScratch<Q, M>) % 16 == 0, "scratch stride must keep 16-byte alignment");
    static constexpr bool ok = true;
};

template <int Q, int M>
__host__ __device__ constexpr size_t smem_bytes_for() {
    static_assert(ScratchChecks<Q, M>::ok, "");
    return (size_t)round_up(Cfg<Q, M>::RBYTES, 128) + (size_t)kWarpsPerCta * sizeof(WarpScratch<Q, M>);
}

// R lookup: value of R at (h-row byte offset hs, column vector c)
template <int Q>
__device__ __forceinline__ int rlookup(const uint8_t *Rs, int hs, int c) {
    if constexpr (Q >= 10) {
        int b = Rs[hs | (c >> 1)];
        return (b >> ((c & 1) << 2)) & 15;
    } else {
        return Rs[hs | c];
    }
}
template <int Q>
__device__ __forceinline__ int hrow_offset(int h) {
    if constexpr (Q >= 10) return h << (Q - 2);   // nibbles: 2^(q-1) entries = 2^(q-2) bytes per row
    else return h << (Q - 1);
}

// ---------------------------------------------------------------- far blocks
// Two-vector: for the groups of middle tile column K, m[r] (lane = column c)
// = max(m[r], A(i,g) + B(g,j) + R[h(i,g)][c(g,j)]), Eq. 3.
template <int Q>
__device__ __forceinline__ void far_block_tv(const FoldParams &P, const SeqDesc &sd, int I, int J, int K, int *m,
                                             WarpScratch<Q, kTwoVector> &ws, const uint8_t *Rs, int lane) {
    using C = Cfg<Q, kTwoVector>;
    constexpr int T = C::T, G = C::G;
    const int Np = sd.Np, NG = Np / Q;
    const uint32_t *RF = P.rf + sd.rf_off;
    const uint32_t *CF = P.cf + sd.cf_off;
    const bool valid = lane < T;
    int B[G], Cv[G];
#pragma unroll
    for (int gl = 0; gl < G; ++gl) {
        int g = K * G + gl;
        uint32_t cf = valid ? __ldcg(CF + (size_t)g * Np + J * T + lane) : 0u;
        uint32_t rf = valid ? __ldcg(RF + (size_t)(I * T + lane) * NG + g) : 0u;
        B[gl] = (int)(cf >> 16);
        Cv[gl] = (int)(cf & C::BMASK);
        ws.rf[gl][lane] = make_int2((int)(rf >> 16), hrow_offset<Q>((int)(rf & C::BMASK)));
    }
    __syncwarp();
#pragma unroll
    for (int gl = 0; gl < G; ++gl) {
#pragma unroll
        for (int r = 0; r < T; ++r) {
            int2 f = ws.rf[gl][r];
            int v = rlookup<Q>(Rs, f.y, Cv[gl]);
            m[r] = max(m[r], f.x + B[gl] + v);
        }
    }
    __syncwarp();
}

// Plain: m[r] holds two packed int16 partial maxima; splits k in [KT+1, KT+T].
static __device__ __forceinline__ void far_block_plain(const FoldParams &P, const SeqDesc &sd, int I, int J, int K,
                                                unsigned *m, WarpScratch<8, kPlain> &ws, int lane) {
    constexpr int T = 32;
    const int Np = sd.Np, PC = sd.PC;
    const int16_t *Drow = P.drow + sd.drow_off;
    const int16_t *Dcol = P.dcol + sd.dcol_off;
    // row strip of row IT+lane, columns KT..KT+31
    const uint4 *src = reinterpret_cast<const uint4 *>(Drow + (size_t)(I * T + lane) * Np + K * T);
    uint4 *dst = reinterpret_cast<uint4 *>(&ws.rows[lane][0]);
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[v] = __ldcg(src + v);
    // own column j = JT+lane, rows KT+1..KT+32 (aligned: index KT+1+kColOff)
    const uint4 *cs = reinterpret_cast<const uint4 *>(Dcol + (size_t)(J * T + lane) * PC + K * T + 1 + kColOff);
    unsigned col[16];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        uint4 w = __ldcg(cs + v);
        col[4 * v + 0] = w.x; col[4 * v + 1] = w.y; col[4 * v + 2] = w.z; col[4 * v + 3] = w.w;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < T; ++r) {
        const uint4 *rw = reinterpret_cast<const uint4 *>(&ws.rows[r][0]);
        unsigned acc = m[r];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            uint4 a = rw[v];
            acc = __viaddmax_s16x2(a.x, col[4 * v + 0], acc);
            acc = __viaddmax_s16x2(a.y, col[4 * v + 1], acc);
            acc = __viaddmax_s16x2(a.z, col[4 * v + 2], acc);
            acc = __viaddmax_s16x2(a.w, col[4 * v + 3], acc);
        }
        m[r] = acc;
    }
    __syncwarp();
}

static __device__ __forceinline__ int hmax2(unsigned a) {
    return max((int)(short)(a & 0xffffu), (int)(short)(a >> 16));
}

// ---------------------------------------------------------------- FAR task
template <int Q, int M>
__device__ void run_far(const FoldParams &P, const SeqDesc &sd, int I, int J, int Ka, int Kb,
                        WarpScratch<Q, M> &ws, const uint8_t *Rs, int lane) {
    constexpr int T = Cfg<Q, M>::T;
    const int NT = sd.NT;
    int *flags = P.flags + sd.flag_off;
    if (Kb < Ka || Ka <= I || Kb >= J) {
        if (lane == 0) atomicCAS(P.error, 0, kErrBadTask);
        return;
    }
    if (!warp_wait_geq(flags + I * NT + Kb, 1, P, lane)) return;
    if (!warp_wait_geq(flags + Ka * NT + J, 1, P, lane)) return;
    if (J - I >= kRing && !warp_wait_geq(flags + I * NT + (J - kRing), 1, P, lane)) return;
    int m[T];
    if constexpr (M == kTwoVector) {
#pragma unroll
        for (int r = 0; r < T; ++r) m[r] = 0;
        for (int K = Ka; K <= Kb; ++K) far_block_tv<Q>(P, sd, I, J, K, m, ws, Rs, lane);
    } else {
        unsigned mp[T];
#pragma unroll
        for (int r = 0; r < T; ++r) mp[r] = 0;
        for (int K = Ka; K <= Kb; ++K) far_block_plain(P, sd, I, J, K, mp, ws, lane);
#pragma unroll
        for (int r = 0; r < T; ++r) m[r] = hmax2(mp[r]);
    }
    int *slot = P.pring + sd.p_off + ((size_t)((J - I) % kRing) * NT + I) * (T * T);
    if (lane < T) {
#pragma unroll
        for (int r = 0; r < T; ++r)
            if (m[r] > 0) atomicMax(slot + r * T + lane, m[r]);
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(P.cnt + sd.cnt_off + I * NT + J, 1);
}

// ---------------------------------------------------------------- NEAR task
template <int Q, int M>
__device__ void run_near(const FoldParams &P, const SeqDesc &sd, int I, int J, int nfar, WarpScratch<Q, M> &ws,
                         const uint8_t *Rs, int lane) {
    using C = Cfg<Q, M>;
    constexpr int T = C::T, G = C::G;
    constexpr bool TV = (M == kTwoVector);
    const int NT = sd.NT, Np = sd.Np, PC = sd.PC;
    const int t = J - I;
    const int IT = I * T, JT = J * T;
    const int c = lane;
    const bool valid = c < T;
    const int j = JT + c;
    int *flags = P.flags + sd.flag_off;
    int16_t *Drow = P.drow + sd.drow_off;
    int16_t *Dcol = P.dcol + sd.dcol_off;
    const uint8_t *codes = P.codes + sd.code_off;

    if (t >= 1) {
        if (!warp_wait_geq(flags + I * NT + (J - 1), 1, P, lane)) return;
        if (!warp_wait_geq(flags + (I + 1) * NT + J, 1, P, lane)) return;
    }
    // far partial max: late blocks K = J-1 and K = I+1 here, the rest from FAR chunks
    int m[T];
    if constexpr (TV) {
#pragma unroll
        for (int r = 0; r < T; ++r) m[r] = 0;
        if (t >= 2) far_block_tv<Q>(P, sd, I, J, J - 1, m, ws, Rs, lane);
        if (t >= 3) far_block_tv<Q>(P, sd, I, J, I + 1, m, ws, Rs, lane);
    } else {
        unsigned mp[T];
#pragma unroll
        for (int r = 0; r < T; ++r) mp[r] = 0;
        if (t >= 2) far_block_plain(P, sd, I, J, J - 1, mp, ws, lane);
        if (t >= 3) far_block_plain(P, sd, I, J, I + 1, mp, ws, lane);
#pragma unroll
        for (int r = 0; r < T; ++r) m[r] = hmax2(mp[r]);
    }
    if (nfar > 0) {
        if (!warp_wait_geq(P.cnt + sd.cnt_off + I * NT + J, nfar, P, lane)) return;
        int *slot = P.pring + sd.p_off + ((size_t)(t % kRing) * NT + I) * (T * T);
        if (valid) {
#pragma unroll
            for (int r = 0; r < T; ++r) {
                m[r] = max(m[r], __ldcg(slot + r * T + c));
                __stcg(slot + r * T + c, 0);   // the ring slot is reused by tile (I, J+kRing)
            }
        }
    }

    // ---- stage inputs
    const int sj = valid ? (int)codes[j] : kPadCode;
    int colv[T + 1];           // colv[r] = D(IT+r, j) once row r is done; colv[T] = D((I+1)T, j)
#pragma unroll
    for (int r = 0; r <= T; ++r) colv[r] = 0;
    if (t >= 1 && valid && (I + 1) * T < Np) colv[T] = ldcg16(Drow + (size_t)((I + 1) * T) * Np + j);
    unsigned Wp[16];           // packed W[c'][c] pairs (off-diagonal tiles)
    if (t >= 1) {
        // diagonal tile (I,I): rows for the residual splits (two-vector) or all column-side splits (plain)
        for (int r = 0; r < T; ++r)
            if (valid) ws.diag[r][c] = (int16_t)ldcg16(Drow + (size_t)(IT + r) * Np + IT + c);
        if constexpr (TV) {
            const int NG = Np / Q;
            for (int r = 0; r < T; ++r)
                if (c < G) ws.drf[r][c] = __ldcg(P.rf + sd.rf_off + (size_t)(IT + r) * NG + I * G + c);
        }
        // left column D(IT+m, JT-1), m = 1..T (pair term of lane 0); rows below JT-1 are 0
        if (valid) {
            int row = IT + 1 + c;   // m = c + 1
            int v = 0;
            if (row <= JT - 1 && row < Np) v = ldcg16(Dcol + (size_t)(JT - 1) * PC + row + kColOff);
            ws.left[c + 1] = (int16_t)v;
        }
        // W column: D(JT+c'+1, j) for c' < c, sentinel otherwise
#pragma unroll
        for (int mm = 0; mm < 16; ++mm) {
            int w0 = kNeg16, w1 = kNeg16;
            int c0 = 2 * mm, c1 = 2 * mm + 1;
            if (valid && c0 < c) w0 = ldcg16(Dcol + (size_t)j * PC + JT + c0 + 1 + kColOff);
            if (valid && c1 < c) w1 = ldcg16(Dcol + (size_t)j * PC + JT + c1 + 1 + kColOff);
            Wp[mm] = (unsigned)(w0 & 0xffff) | ((unsigned)w1 << 16);
        }
    } else {
#pragma unroll
        for (int mm = 0; mm < 16; ++mm) Wp[mm] = 0;
    }
    if (c == 0) ws.left[0] = 0;
    __syncwarp();

    const unsigned long long pair64 = P.pair64;
    int below = colv[T];       // D(i+1, j) for the current row i
    unsigned vhist = 0;        // vertical differences, newest in bit 0
    int colB[G], colC[G];
#pragma unroll
    for (int gl = 0; gl < G; ++gl) { colB[gl] = 0; colC[gl] = 0; }
    const int NG = TV ? Np / Q : 1;

#pragma unroll
    for (int r = T - 1; r >= 0; --r) {
        const int i = IT + r;
        const int si = (int)codes[i];
        const unsigned rowbits = (unsigned)(pair64 >> (8 * si)) & 0xffu;
        // D(i+1, j-1): lane c-1's previous row; lane 0 reads the left column
        int bl = __shfl_up_sync(FULL, below, 1);
        if (c == 0) bl = (r == T - 1) ? ((t >= 1 && J >= 1) ? (int)ws.left[T] : 0) : (int)ws.left[r + 1];
        const int pb = (int)((rowbits >> sj) & 1u);
        int y;
        if (t == 0) {
            y = (c > r) ? pb + bl : (c == r ? 0 : kNeg16);
        } else {
            y = max(pb + bl, m[r]);
            if constexpr (TV) {
                const int ce = (r + Q - 1) / Q * Q;
                // residual splits k in [i+1, IT+ce]: D(i,k-1) from tile (I,I), D(k,j) from this column
#pragma unroll
                for (int kk = r + 1; kk <= ce; ++kk) y = max(y, (int)ws.diag[r][kk - 1] + colv[kk]);
                // full groups of tile column I with g*q >= i (Eq. 3)
#pragma unroll
                for (int gl = ce / Q; gl < G; ++gl) {
                    uint32_t f = ws.drf[r][gl];
                    int v = rlookup<Q>(Rs, hrow_offset<Q>((int)(f & C::BMASK)), colC[gl]);
                    y = max(y, (int)(f >> 16) + colB[gl] + v);
                }
            } else {
                // every split with D(k,j) in this tile column: k in [i+1, IT+T]
#pragma unroll
                for (int kk = r + 1; kk <= T; ++kk) y = max(y, (int)ws.diag[r][kk - 1] + colv[kk]);
            }
        }
        if (!valid) y = kNeg16;
        // closure over the row: D_c = max(Y_c, max_{c'<c} Y_c' + W[c'][c])
        ws.y[c] = (int16_t)y;
        __syncwarp();
        unsigned acc = 0;
        const uint4 *yp = reinterpret_cast<const uint4 *>(ws.y);
        if (t == 0) {
            // W from this (diagonal) tile's own column: D(IT+c'+1, j), valid for rows already done
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                uint4 a = yp[v];
                unsigned aw[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    int c0 = 8 * v + 2 * e, c1 = c0 + 1;
                    int w0 = (c0 < c && c0 + 1 <= T) ? colv[c0 + 1 <= T ? c0 + 1 : T] : kNeg16;
                    int w1 = (c1 < c && c1 + 1 <= T) ? colv[c1 + 1 <= T ? c1 + 1 : T] : kNeg16;
                    unsigned wp = (unsigned)(w0 & 0xffff) | ((unsigned)w1 << 16);
                    acc = __viaddmax_s16x2(aw[e], wp, acc);
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                uint4 a = yp[v];
                acc = __viaddmax_s16x2(a.x, Wp[4 * v + 0], acc);
                acc = __viaddmax_s16x2(a.y, Wp[4 * v + 1], acc);
                acc = __viaddmax_s16x2(a.z, Wp[4 * v + 2], acc);
                acc = __viaddmax_s16x2(a.w, Wp[4 * v + 3], acc);
            }
        }
        __syncwarp();
        int d = max(y, hmax2(acc));
        if (t == 0 && c < r) d = 0;
        if (!valid) d = 0;
        // ---- features
        const int vb = d - colv[r + 1];   // vertical difference D(i,j) - D(i+1,j)
        vhist = (vhist << 1) | (unsigned)(vb & 1);
        colv[r] = d;
        below = d;
        if (valid) ws.tile[r][c] = (int16_t)d;
        if constexpr (TV) {
            if (r >= 1 && (r - 1) % Q == 0) {
                const int gl = (r - 1) / Q;   // group rows gl*q+1 .. gl*q+q complete
                colB[gl] = d;
                colC[gl] = (int)(vhist & C::BMASK);
                if (valid) P.cf[sd.cf_off + (size_t)(I * G + gl) * Np + j] = ((uint32_t)d << 16) | (vhist & C::BMASK);
            }
            const int dl = __shfl_up_sync(FULL, d, 1);
            const unsigned hb = __ballot_sync(FULL, (d - dl) == 1);
            const int a = __shfl_sync(FULL, d, (c < G) ? c * Q : 0);
            if (c < G)
                P.rf[sd.rf_off + (size_t)i * NG + J * G + c] = ((uint32_t)a << 16) | ((hb >> (c * Q + 1)) & C::BMASK);
        }
    }
    __syncwarp();
    // ---- store both copies: row-major rows (coalesced over lanes = columns) ...
    if (valid) {
#pragma unroll 4
        for (int r = 0; r < T; ++r) Drow[(size_t)(IT + r) * Np + j] = ws.tile[r][c];
    }
    // ... and column-major columns (lane = row)
    if (lane < T) {
#pragma unroll 4
        for (int cc = 0; cc < T; ++cc) Dcol[(size_t)(JT + cc) * PC + IT + lane + kColOff] = ws.tile[lane][cc];
    }
    // answer D(0, n-1)
    if (I == 0 && J == NT - 1) {
        int cn = (sd.n - 1) - JT;
        if (sd.n >= 1 && lane == cn) P.results[sd.result_index] = (sd.n >= 2) ? (int)ws.tile[0][cn] : 0;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + I * NT + J, 1);
}

// ---------------------------------------------------------------- kernel
template <int Q, int M>
__global__ void __launch_bounds__(kThreads, 1) fold_kernel(FoldParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    using C = Cfg<Q, M>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *Rs = smem;
    if constexpr (C::RBYTES > 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.rtab);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        // the device copy of R is padded to a multiple of 256 bytes, so rounding up stays in bounds
        for (int v = threadIdx.x; v < (C::RBYTES + 15) / 16; v += blockDim.x) dst[v] = __ldg(src + v);
    }
    __syncthreads();
    WarpScratch<Q, M> &ws =
        *reinterpret_cast<WarpScratch<Q, M> *>(smem + round_up(C::RBYTES, 128) + warp * sizeof(WarpScratch<Q, M>));
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(P.queue_head, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= P.ntasks) break;
        if (*(volatile int *)P.error != 0) break;
        const int4 tk = P.tasks[idx];
        const SeqDesc sd = P.seqs[tk.x];
        const int I = task_I(tk.y), J = task_J(tk.y);
        if (task_type(tk.y) == kTaskNear) run_near<Q, M>(P, sd, I, J, tk.z, ws, Rs, lane);
        else run_far<Q, M>(P, sd, I, J, tk.z, tk.w, ws, Rs, lane);
    }
}

template <int Q, int M>
inline cudaError_t launch_q(const FoldParams &p, int grid, cudaStream_t st) {
    size_t sm = smem_bytes_for<Q, M>();
    cudaError_t e = cudaFuncSetAttribute(fold_kernel<Q, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    fold_kernel<Q, M><<<grid, kThreads, sm, st>>>(p);
    return cudaGetLastError();
}

template <int Q, int M>
inline int blocks_per_sm_q() {
    int nb = 0;
    size_t sm = smem_bytes_for<Q, M>();
    if (cudaFuncSetAttribute(fold_kernel<Q, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fold_kernel<Q, M>, kThreads, sm) != cudaSuccess) return 0;
    return nb;
}

}  // namespace fold
