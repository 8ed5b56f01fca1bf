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
static __device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// relaxed gpu-scope add without a return value (a release when a fence.acq_rel precedes it)
static __device__ __forceinline__ void red_add(int *p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ void st_relaxed(int *p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
static __device__ __forceinline__ unsigned smid() {
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// Lane 0 waits (bounded) until *p >= target; the verdict is broadcast.  On
// timeout the error word is set; any error seen makes every worker stop.
static __device__ __noinline__ bool wait_geq_impl(const int *p, int target, int *error, long long timeout_ns, int lane) {
    int ok = 1;
    if (lane == 0) {
        if (ld_acquire(p) < target) {
            // poll without sleeping for the first 2 us (dependencies usually resolve within a few
            // L2 round trips), then back off to at most 256 ns between polls
            const unsigned long long t0 = gtimer();
            unsigned ns = 0;
            for (;;) {
                if (ns) __nanosleep(ns);
                if (ld_acquire(p) >= target) break;
                if (*(volatile int *)error != 0) { ok = 0; break; }
                const long long el = (long long)(gtimer() - t0);
                if (el > 2000) ns = ns ? (ns < 256 ? 2 * ns : 256) : 32;
                if (el > timeout_ns) {
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
// Up to three tile flags (null = none) acquired by lanes 0-2 at once, so the usual case (all set)
// costs one round trip; the warp barrier orders every lane's later loads after the acquires (as in
// wait_geq_impl).  A flag not yet set is then awaited by warp_wait_geq.
static __device__ __forceinline__ bool warp_wait_flags(const int *f0, const int *f1, const int *f2, const FoldParams &P,
                                                       int lane) {
    const int *mine = lane == 0 ? f0 : lane == 1 ? f1 : lane == 2 ? f2 : nullptr;
    const unsigned miss = __ballot_sync(FULL, mine != nullptr && ld_acquire(mine) < 1);
    __syncwarp();
    if ((miss & 1u) && !warp_wait_geq(f0, 1, P, lane)) return false;
    if ((miss & 2u) && !warp_wait_geq(f1, 1, P, lane)) return false;
    if ((miss & 4u) && !warp_wait_geq(f2, 1, P, lane)) return false;
    return true;
}

// shared-memory flags between the warps of one CTA (column mode)
static __device__ __forceinline__ int ld_acquire_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
static __device__ __forceinline__ void st_release_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
// Lane 0 waits (bounded) until the shared word *p >= target; the error word and the clock are
// checked every 32 polls so that a poll costs one shared load.
static __device__ __noinline__ bool wait_smem_geq_slow(const int *p, int target, int *error, long long timeout_ns, int lane) {
    int ok = 1;
    if (lane == 0 && ld_acquire_cta(p) < target) {
        const unsigned long long t0 = gtimer();
        for (unsigned it = 1;; ++it) {
            if (ld_acquire_cta(p) >= target) break;
            if ((it & 31u) == 0) {
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
static __device__ __forceinline__ bool wait_smem_geq(const int *p, int target, int *error, long long timeout_ns, int lane) {
    int v = 0;
    if (lane == 0) v = ld_acquire_cta(p);
    if (__shfl_sync(FULL, v, 0) >= target) {
        __syncwarp();
        return true;
    }
    return wait_smem_geq_slow(p, target, error, timeout_ns, lane);
}

// max into global memory without returning the old value (a reduction, not an atomic: nothing
// comes back to the SM; the fence that follows the merges orders them before the chunk count)
static __device__ __forceinline__ void red_max(int *p, int v) {
    asm volatile("red.relaxed.gpu.global.max.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bulk reduction of a 16-byte-aligned shared buffer into global memory by the async proxy (one
// instruction instead of one red per element); the shared source must be made visible to the async
// proxy first (fence_proxy_async_smem by every writing thread), the destination's earlier generic
// writes that the issuing thread has acquired are ordered before it by fence_proxy_async_global,
// and the async proxy's global writes are fenced into the generic proxy (fence_proxy_async_global
// again, after completion) before a release publishes them.
static __device__ __forceinline__ void bulk_red_max_s32(int *gdst, const int *ssrc, unsigned bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.max.s32 [%0], [%1], %2;"
                 ::"l"(gdst), "r"((unsigned)__cvta_generic_to_shared(ssrc)), "r"(bytes) : "memory");
}
static __device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared sources of every committed bulk operation have been read (they may be rewritten)
static __device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// every committed bulk operation is complete
static __device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
static __device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// 16-byte global -> shared copies that bypass L1 (both addresses 16-byte aligned)
static __device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
static __device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// two-vector: residual splits per row of a tile (the window of rows below it)
template <int Q>
constexpr int NW_RES = Q > 1 ? Q - 1 : 1;

// per-warp shared scratch
template <int Q, int M>
struct __align__(16) WarpScratch {
    static constexpr int T = Cfg<Q, M>::T;
    static constexpr int G = Cfg<Q, M>::G;
    static constexpr bool PL = (M == kPlain);
    static constexpr int LR = PL ? 32 : 1;         // plain: late-block row strips
    static constexpr int LF = PL ? 1 : T;          // two-vector: late-block row features
    static constexpr int SS = strip_of(Q, M);
    static constexpr int DS = PL ? 40 : 32;    // diagonal-tile row stride: 16-byte rows (uint4 / cp.async)
    static constexpr int NWP = (Q > 2 ? Q : 2) / 2;   // two-vector residual window: Q-1 values in pairs
    static constexpr int NWPA = (NWP + 3) / 4 * 4;     // ... padded to 16-byte rows
    static constexpr int GA = (G + 3) / 4 * 4;         // groups padded to 16-byte rows
    // column mode copies a tile's P slot into shared memory with 16-byte cp.async (T*T a multiple of
    // four ints; left out where the per-block shared memory would not hold it)
    static constexpr bool PB = (T * T) % 4 == 0 && !(M == kTwoVector && Q >= 10);
    union {
        struct {                       // chunk tasks
            int2 rf[G][32];            // STRIP staging (two-vector): (A in both halves, h-row byte offset)
            alignas(16) uint32_t rfw[PL ? 1 : 32][PL ? 4 : GA];  // FAR staging (two-vector): per row,
                                       // (A << 16 | R-row offset) of each group
            uint32_t scv[PL ? 1 : G][PL ? 1 : SS + SS / 2][32];  // STRIP staging (two-vector): per group,
                                       // the lane's column bits for SS columns and SS/2 packed base pairs
            alignas(16) int16_t rows[LR][32];  // FAR staging (plain): row strips (uint4 access)
        };
        struct {                       // column mode (its warps run no chunk tasks)
            int16_t tile1[T + 1][33];  // second output buffer: tiles alternate between tile and tile1
            uint32_t rfo[2][LF][G];    // row features of the last two tiles (two-vector), read by the
                                       // warp of the next column
            alignas(16) int pbuf[PB ? T * T : 4];  // the tile's P slot (far partial max), row-major
        };
    };
    alignas(16) int16_t lrow[2][LR][32];  // NEAR late blocks (plain): rows of tiles (I,J-1), (I,I+1)
    alignas(16) uint32_t colpk[PL ? 16 : 1][32];  // NEAR (plain): (D(IT+2m+1,j), D(IT+2m+2,j)) pairs, per lane
    alignas(16) uint32_t lrf[2][LF][G];  // NEAR late blocks (two-vector): row features of (I,J-1), (I,I+1)
    alignas(16) uint32_t cbc[32][PL ? 4 : GA];  // NEAR (two-vector): (B << 16 | bits) of the lane's column
                                       // groups, lane-major (one 16-byte load per four groups)
    alignas(16) int16_t diag[T][DS];   // diagonal tile (I,I) rows
    alignas(16) uint32_t gw[PL ? 1 : T][PL ? 4 : GA];  // NEAR (two-vector): per row of the diagonal tile
                                       // and group, (A << 16) | R-row offset (h for nibble tables), with
                                       // A = -32768 for groups not complete below that row
    alignas(16) uint32_t rpk[PL ? 1 : T][PL ? 4 : NWPA];  // NEAR (two-vector): per row, the residual
                                       // splits' D(i, k-1) as int16 pairs, -32768 where k is not a
                                       // residual split of the row
    int16_t pm[T][32];                 // far partial max of each row (lane = column)
    alignas(16) int16_t y[2][32];      // closure exchange, double-buffered (read back as uint4)
    int16_t left[T + 2];               // D(IT+m, JT-1)
    int16_t tile[T + 1][33];           // output tile; row T holds D((I+1)T, j); 33 columns so every lane's
                                       // index (also lanes >= T) stays inside the array
    int produced;                      // column mode: tiles of this column published in shared memory
    int consumed;                      // column mode, written by the next column's warp: tiles it has read
};

// every vector-accessed member must sit on a 16-byte boundary
template <int Q, int M>
struct ScratchChecks {
    using WS = WarpScratch<Q, M>;
    static_assert(offsetof(WS, y) % 16 == 0, "y must be 16-byte aligned");
    static_assert(offsetof(WS, rows) % 16 == 0, "rows must be 16-byte aligned");
    static_assert(offsetof(WS, rfw) % 16 == 0, "rfw rows are read as uint4");
    static_assert(offsetof(WS, rf) % 16 == 0, "rf row pairs are read as uint4");
    static_assert(offsetof(WS, lrow) % 16 == 0, "lrow must be 16-byte aligned");
    static_assert(offsetof(WS, pbuf) % 16 == 0, "pbuf is written by 16-byte cp.async");
    static_assert(offsetof(WS, lrf) % 16 == 0, "lrf must be 16-byte aligned");
    static_assert(offsetof(WS, cbc) % 16 == 0 && offsetof(WS, gw) % 16 == 0 && offsetof(WS, rpk) % 16 == 0,
                  "cbc, gw and rpk rows are read as uint4");
    static_assert(offsetof(WS, diag) % 16 == 0 && (WS::DS * 2) % 16 == 0, "diag rows 16-byte aligned");
    static_assert(sizeof(WarpScratch<Q, M>) % 16 == 0, "scratch stride must keep 16-byte alignment");
    static constexpr bool ok = true;
};

// partially memoised R (two-vector, byte tables): one bit per horizontal vector, set once its row
// is tabulated in this CTA
template <int Q, int M>
__host__ __device__ constexpr int memo_words() {
    return (M == kTwoVector && !Cfg<Q, M>::NIB) ? ((1 << (Q - 1)) + 31) / 32 : 0;
}
template <int Q, int M>
__host__ __device__ constexpr size_t memo_offset() {
    return (size_t)round_up(Cfg<Q, M>::RBYTES, 128) + (size_t)kWarpsPerCta * sizeof(WarpScratch<Q, M>);
}

template <int Q, int M>
__host__ __device__ constexpr size_t smem_bytes_for() {
    static_assert(ScratchChecks<Q, M>::ok, "");
    static_assert(memo_offset<Q, M>() + 16 * (size_t)((memo_words<Q, M>() + 3) / 4) <= 227 * 1024,
                  "R table plus per-warp scratch must fit the 227 KB per-block shared memory of sm_103a");
    return memo_offset<Q, M>() + 16 * (size_t)((memo_words<Q, M>() + 3) / 4);
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

// Partially memoised R (Section 3.2): before a warp stages features for lookups, every row R[h][*]
// they use must be tabulated in this CTA.  Lanes whose h has no row yet ask; the warp fills the asked
// rows one at a time (lane l computes the entries c = l, l+32, ... by the Section 3.1 routine, the
// best prefix sum of h_p - c_p over p), then lane 0 publishes the row's bit with a CTA-scope release;
// a reader sees the bit with an acquire load before it reads the row.  Two warps may fill the same
// row at once: they write the same bytes.
template <int Q, int M>
__device__ __noinline__ void memo_fill(uint8_t *Rs, unsigned ask_mask, unsigned h, int lane) {
    constexpr int NB = Q - 1;
    unsigned *bits = reinterpret_cast<unsigned *>(Rs + memo_offset<Q, M>());
    unsigned m = ask_mask;
    while (m) {
        const unsigned hr = __shfl_sync(FULL, h, __ffs(m) - 1);
        for (int c = lane; c < (1 << NB); c += 32) {
            int best = 0, sum = 0;
#pragma unroll
            for (int p = 1; p <= NB; ++p) {
                sum += (int)((hr >> (p - 1)) & 1u) - (int)(((unsigned)c >> (p - 1)) & 1u);
                best = max(best, sum);
            }
            Rs[(hr << NB) | (unsigned)c] = (uint8_t)best;
        }
        __syncwarp();
        if (lane == 0)
            asm volatile("red.release.cta.shared::cta.or.b32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bits + (hr >> 5))),
                         "r"(1u << (hr & 31)) : "memory");
        m &= ~__ballot_sync(FULL, (m >> lane & 1u) && h == hr);
    }
    __syncwarp();
}
template <int Q, int M, bool MEMO>
__device__ __forceinline__ void memo_ensure(const uint8_t *Rs, unsigned h, bool need, int lane) {
    if constexpr (MEMO && memo_words<Q, M>() > 0) {
        const unsigned *bits = reinterpret_cast<const unsigned *>(Rs + memo_offset<Q, M>());
        const bool ask = need && !((ld_acquire_cta(reinterpret_cast<const int *>(bits + (h >> 5))) >> (h & 31)) & 1);
        const unsigned m = __ballot_sync(FULL, ask);
        if (m) memo_fill<Q, M>(const_cast<uint8_t *>(Rs), m, h, lane);
    }
}

// One full group's candidate of Eq. 3, A + B + R[h][c], scaled by 2^16 (the low half is not zero):
// w = (A << 16) | R-row offset of h (h itself for nibble tables), cb = (B << 16) | c.  A and B are
// D values of two disjoint pieces of [i, j], so A + B <= (j-i+1)/2 < 2^15 and one 32-bit add gives
// A + B in the high half (also for A = -32768, which stays negative with B >= 0) and the R index in
// the low half (the offset and c share no bits).  Candidates compare as signed integers.
template <int Q>
__device__ __forceinline__ int group_term(const uint8_t *Rs, uint32_t w, uint32_t cb) {
    if constexpr (Q >= 10) {
        constexpr unsigned BM = (1u << (Q - 1)) - 1;
        const uint32_t s = w + (cb & 0xffff0000u);
        const int v = rlookup<Q>(Rs, hrow_offset<Q>((int)(w & BM)), (int)(cb & BM));
        return (int)(s + ((uint32_t)v << 16));
    } else {
        const uint32_t s = w + cb;
        return (int)(s + ((uint32_t)Rs[s & 0xffffu] << 16));
    }
}

// A row feature (A << 16 | h) as the word group_term takes: h replaced by its R-row offset
// (kept as h for nibble tables, whose offsets need more than 16 bits).
template <int Q>
__device__ __forceinline__ uint32_t group_word(uint32_t f) {
    constexpr unsigned BM = (1u << (Q - 1)) - 1;
    if constexpr (Q >= 10) return f;
    else return (f & 0xffff0000u) | (uint32_t)hrow_offset<Q>((int)(f & BM));
}

// ---------------------------------------------------------------- far blocks
// Two-vector, a chunk of middle blocks [Ka, Kb] of tile (I,J): for each group g of the blocks,
// m[r] (lane = column c) = max(m[r], A(i,g) + B(g,j) + R[h(i,g)][c(g,j)]), Eq. 3.  The rows'
// features go to shared memory as words (A << 16 | R-row offset), four groups per 16-byte
// broadcast load; the lane's column feature (B << 16 | c) is used as loaded.  The features of
// block K+1 are loaded while block K is evaluated, so each block's L2 latency overlaps the
// previous block.  m[] is kept scaled by 2^16 inside (see group_term).
template <int Q, bool MEMO>
__device__ __forceinline__ void far_chunk_tv(const FoldParams &P, const SeqDesc &sd, int I, int J, int Ka, int Kb,
                                             int *m, WarpScratch<Q, kTwoVector> &ws, const uint8_t *Rs, int lane) {
    using C = Cfg<Q, kTwoVector>;
    using WS = WarpScratch<Q, kTwoVector>;
    constexpr int T = C::T, G = C::G;
    const int Np = sd.Np, NG = Np / Q;
    const uint32_t *RF = P.rf + sd.rf_off;
    const uint32_t *CF = P.cf + sd.cf_off;
    const bool valid = lane < T;
    uint32_t cfn[G], rfn[G];
#pragma unroll
    for (int gl = 0; gl < G; ++gl) {
        const int g = Ka * G + gl;
        cfn[gl] = valid ? __ldcg(CF + (size_t)g * Np + J * T + lane) : 0u;
        rfn[gl] = valid ? __ldcg(RF + (size_t)(I * T + lane) * NG + g) : 0u;
    }
#pragma unroll
    for (int r = 0; r < T; ++r) m[r] = (int)((unsigned)m[r] << 16);
    for (int K = Ka; K <= Kb; ++K) {
        uint32_t cb[G];
        uint32_t w[WS::GA];
#pragma unroll
        for (int gl = 0; gl < WS::GA; ++gl) {
            const uint32_t f = gl < G ? rfn[min(gl, G - 1)] : 0u;
            w[gl] = (f & 0xffff0000u) | (C::NIB ? (f & C::BMASK) : (uint32_t)hrow_offset<Q>((int)(f & C::BMASK)));
        }
#pragma unroll
        for (int gl = 0; gl < G; ++gl) cb[gl] = cfn[gl];
#pragma unroll
        for (int gl = 0; gl < G; ++gl) memo_ensure<Q, kTwoVector, MEMO>(Rs, rfn[gl] & C::BMASK, valid, lane);
#pragma unroll
        for (int g4 = 0; g4 < WS::GA / 4; ++g4)
            reinterpret_cast<uint4 *>(&ws.rfw[lane][0])[g4] = make_uint4(w[4 * g4], w[4 * g4 + 1], w[4 * g4 + 2], w[4 * g4 + 3]);
        if (K < Kb) {   // prefetch the next block
#pragma unroll
            for (int gl = 0; gl < G; ++gl) {
                const int g = (K + 1) * G + gl;
                cfn[gl] = valid ? __ldcg(CF + (size_t)g * Np + J * T + lane) : 0u;
                rfn[gl] = valid ? __ldcg(RF + (size_t)(I * T + lane) * NG + g) : 0u;
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < T; ++r) {
#pragma unroll
            for (int g4 = 0; g4 < WS::GA / 4; ++g4) {
                const uint4 w4 = reinterpret_cast<const uint4 *>(&ws.rfw[r][0])[g4];
                if (4 * g4 + 0 < G) m[r] = max(m[r], group_term<Q>(Rs, w4.x, cb[min(4 * g4 + 0, G - 1)]));
                if (4 * g4 + 1 < G) m[r] = max(m[r], group_term<Q>(Rs, w4.y, cb[min(4 * g4 + 1, G - 1)]));
                if (4 * g4 + 2 < G) m[r] = max(m[r], group_term<Q>(Rs, w4.z, cb[min(4 * g4 + 2, G - 1)]));
                if (4 * g4 + 3 < G) m[r] = max(m[r], group_term<Q>(Rs, w4.w, cb[min(4 * g4 + 3, G - 1)]));
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < T; ++r) m[r] >>= 16;
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

// max of N values as a balanced tree (short dependency chains)
template <int N>
__device__ __forceinline__ int tree_max(int (&v)[N]) {
    int w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = v[k];
#pragma unroll
    for (int span = 1; span < N; span *= 2) {
#pragma unroll
        for (int k = 0; k + span < N; k += 2 * span) w[k] = max(w[k], w[k + span]);
    }
    return w[0];
}

static __device__ __forceinline__ int hmax2(unsigned a) {
    return max((int)(short)(a & 0xffffu), (int)(short)(a >> 16));
}

// serving ring: lane 0 waits (bounded) until index idx is published or the host has stopped; the
// verdict (1: no task for this claim) is broadcast.  A free function with scalar arguments, so that
// neither the task claim nor the kernel parameters need an address.
static __device__ __noinline__ int ring_wait(const int *tail, const int *stop, int *error, long long timeout_ns, int idx,
                                             int lane) {
    int st = 0;
    if (lane == 0 && ld_acquire(tail) <= idx) {
        const unsigned long long t0 = gtimer();
        unsigned ns = 0;
        for (;;) {
            if (ld_acquire(tail) > idx) break;
            if (ld_acquire(stop) != 0) {
                if (ld_acquire(tail) > idx) break;
                st = 1;
                break;
            }
            if (*(volatile int *)error != 0) { st = 1; break; }
            if ((long long)(gtimer() - t0) > timeout_ns) {
                atomicCAS(error, 0, kErrTimeout);
                st = 1;
                break;
            }
            __nanosleep(ns);
            ns = ns ? (ns < 1024 ? 2 * ns : 1024) : 64;
        }
    }
    st = __shfl_sync(FULL, st, 0);
    __syncwarp();
    return st;
}

// The queue's next task for a worker: claimed while the worker finishes its current chunk, right
// after the chunk's merges are issued, so that the claim's round trips (queue atomic, task load)
// overlap the merges' completion.  The claim comes only the merge's duration early, so tasks still
// start in about list order.
struct NextTask {
    int *qhead;
    int qbase, qlimit;
    const int4 *tasks;
    int idx;
    int4 tk;
    bool have;
    bool stopped;  // serving ring: the host stopped publishing and this claim has no task
    int pending;   // lane 0: the queue atomic's result, read by finish()
    int ring_cap;  // serving ring (see FoldParams), 0 otherwise
    const int *ring_tail, *ring_stop;
    int *ring_progress, *error;
    long long timeout_ns;
    // the queue atomic goes out here; its result is read by finish()
    __device__ __forceinline__ void start(int lane) {
        if (lane == 0) pending = atomicAdd(qhead, 1);
    }
    __device__ __forceinline__ void finish(int lane) {
        const int i = qbase + __shfl_sync(FULL, lane == 0 ? pending : 0, 0);
        idx = i;
        // serving ring: the task is fetched by fetch() once the current task is complete (a chunk
        // claims its successor before it counts itself done, and the successor may not be published)
        tk = (ring_cap == 0 && i < qlimit) ? tasks[i] : make_int4(0, 0, 0, 0);
        have = true;
    }
    // serving ring: wait until the claimed task is published (or the host stopped), then load it
    __device__ __forceinline__ void fetch(int lane) {
        if (ring_cap == 0) return;
        stopped = ring_wait(ring_tail, ring_stop, error, timeout_ns, idx, lane) != 0;
        tk = stopped ? make_int4(0, 0, 0, 0) : __ldcg(tasks + (idx % ring_cap));
        if (lane == 0 && (idx & 255) == 0) *(volatile int *)ring_progress = idx;
    }
    __device__ __forceinline__ void claim(int lane) {
        start(lane);
        finish(lane);
    }
};

// ---------------------------------------------------------------- FAR task
template <int Q, int M, bool MEMO>
__device__ __forceinline__ long long run_far(const FoldParams &P, const SeqDesc &sd, int I, int J, int Ka, int Kb,
                        WarpScratch<Q, M> &ws, const uint8_t *Rs, int lane, long long *tdeps, NextTask &nt) {
    constexpr int T = Cfg<Q, M>::T;
    const int NT = sd.NT;
    int *flags = P.flags + sd.flag_off;
    if (Kb < Ka || Ka <= I || Kb >= J) {
        if (lane == 0) atomicCAS(P.error, 0, kErrBadTask);
        return 0;
    }
    // row strip (I, Kb), column strip (Ka, J) and, past the P ring's depth, the tile whose slot this reuses
    if (!warp_wait_flags(flags + I * NT + Kb, flags + Ka * NT + J, J - I >= kRing ? flags + I * NT + (J - kRing) : nullptr,
                         P, lane))
        return 0;
    if (P.trace) tdeps[0] = (long long)gtimer();
    int m[T];
    if constexpr (M == kTwoVector) {
#pragma unroll
        for (int r = 0; r < T; ++r) m[r] = 0;
        far_chunk_tv<Q, MEMO>(P, sd, I, J, Ka, Kb, m, ws, Rs, lane);
    } else {
        unsigned mp[T];
#pragma unroll
        for (int r = 0; r < T; ++r) mp[r] = 0;
        for (int K = Ka; K <= Kb; ++K) far_block_plain(P, sd, I, J, K, mp, ws, lane);
#pragma unroll
        for (int r = 0; r < T; ++r) m[r] = hmax2(mp[r]);
    }
    const long long tdone = P.trace ? (long long)gtimer() : 0;
    nt.start(lane);
    int *slot = P.pring + sd.p_off + ((size_t)((J - I) % kRing) * NT + I) * (T * T);
    if constexpr (WarpScratch<Q, M>::PB) {
        // the partial maximum is staged in shared memory (pbuf shares its bytes with the chunk
        // staging, free once the lookups are done) and merged by one bulk reduction; lane 0 waits
        // for it, fences the async proxy's writes and publishes the count
        __syncwarp();
        if (lane < T) {
#pragma unroll
            for (int r = 0; r < T; ++r) ws.pbuf[r * T + lane] = m[r];
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            // the slot's zeroing by the tile that used it before (acquired with the input flags, by
            // the generic proxy) is ordered before the async proxy's reduction into it
            fence_proxy_async_global();
            bulk_red_max_s32(slot, ws.pbuf, (unsigned)(T * T * sizeof(int)));
            bulk_commit();
        }
        nt.finish(lane);
        if (lane == 0) {
            bulk_wait_all();
            fence_proxy_async_global();
            fence_acq_rel();   // releases the merge with the relaxed count below
            red_add(P.cnt + sd.cnt_off + I * NT + J, 1);
        }
        __syncwarp();
    } else {
        if (lane < T) {
#pragma unroll
            for (int r = 0; r < T; ++r)
                if (m[r] > 0) red_max(slot + r * T + lane, m[r]);
        }
        nt.finish(lane);
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(P.cnt + sd.cnt_off + I * NT + J, 1);
    }
    return tdone;
}

// ---------------------------------------------------------------- STRIP chunks
// Two-vector strip: S tiles (I, J0..J0+S-1) at once, lane = column c of each.
// For every (row, group) the warp-uniform row feature (A duplicated into both
// 16-bit halves, h-row offset) is one broadcast load that serves S lookups;
// two columns share one packed 16x2 accumulator (A + B + R <= n/2 < 2^15, so
// the halves never carry into each other).
template <int Q, int S, bool MEMO>
__device__ __forceinline__ void far_strip_tv(const FoldParams &P, const SeqDesc &sd, int I, int J0, int Seff, int Ka,
                                             int Kb, unsigned (&m2)[S / 2][Cfg<Q, kTwoVector>::T],
                                             WarpScratch<Q, kTwoVector> &ws, const uint8_t *Rs, int lane) {
    using C = Cfg<Q, kTwoVector>;
    constexpr int T = C::T, G = C::G;
    const int Np = sd.Np, NG = Np / Q;
    const uint32_t *RF = P.rf + sd.rf_off;
    const uint32_t *CF = P.cf + sd.cf_off;
    const bool lv = lane < T;
    uint32_t cfn[S][G], rfn[G];
#pragma unroll
    for (int gl = 0; gl < G; ++gl) {
        const int g = Ka * G + gl;
#pragma unroll
        for (int s = 0; s < S; ++s) cfn[s][gl] = (lv && s < Seff) ? __ldcg(CF + (size_t)g * Np + (J0 + s) * T + lane) : 0u;
        rfn[gl] = lv ? __ldcg(RF + (size_t)(I * T + lane) * NG + g) : 0u;
    }
    for (int K = Ka; K <= Kb; ++K) {
#pragma unroll
        for (int gl = 0; gl < G; ++gl) {
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) ws.scv[gl][s2][lane] = cfn[s2][gl] & C::BMASK;
#pragma unroll
            for (int p2 = 0; p2 < S / 2; ++p2)
                ws.scv[gl][S + p2][lane] = (cfn[2 * p2][gl] >> 16) | (cfn[2 * p2 + 1][gl] & 0xffff0000u);
            ws.rf[gl][lane] = make_int2((int)((rfn[gl] >> 16) * 0x10001u), hrow_offset<Q>((int)(rfn[gl] & C::BMASK)));
            memo_ensure<Q, kTwoVector, MEMO>(Rs, rfn[gl] & C::BMASK, lv, lane);
        }
        if (K < Kb) {   // prefetch the next block
#pragma unroll
            for (int gl = 0; gl < G; ++gl) {
                const int g = (K + 1) * G + gl;
#pragma unroll
                for (int s2 = 0; s2 < S; ++s2)
                    cfn[s2][gl] = (lv && s2 < Seff) ? __ldcg(CF + (size_t)g * Np + (J0 + s2) * T + lane) : 0u;
                rfn[gl] = lv ? __ldcg(RF + (size_t)(I * T + lane) * NG + g) : 0u;
            }
        }
        __syncwarp();
        // one group at a time (a runtime loop keeps the live register set small)
#pragma unroll 1
        for (int gl = 0; gl < G; ++gl) {
            int cv[S];
            unsigned b2[S / 2];
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) cv[s2] = (int)ws.scv[gl][s2][lane];
#pragma unroll
            for (int p2 = 0; p2 < S / 2; ++p2) b2[p2] = ws.scv[gl][S + p2][lane];
            // two rows' features per 16-byte broadcast load
#pragma unroll
            for (int r2 = 0; r2 < (T + 1) / 2; ++r2) {
                const uint4 f2 = reinterpret_cast<const uint4 *>(&ws.rf[gl][0])[r2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int r = 2 * r2 + u;
                    if (r >= T) break;
                    const unsigned fx = u ? f2.z : f2.x;
                    const int fy = (int)(u ? f2.w : f2.y);
#pragma unroll
                    for (int p2 = 0; p2 < S / 2; ++p2) {
                        const unsigned v0 = (unsigned)rlookup<Q>(Rs, fy, cv[2 * p2]);
                        const unsigned v1 = (unsigned)rlookup<Q>(Rs, fy, cv[2 * p2 + 1]);
                        const unsigned t = fx + b2[p2] + (v1 * 65536u + v0);
                        m2[p2][r] = __vmaxs2(m2[p2][r], t);
                    }
                }
            }
        }
        __syncwarp();
    }
}

// Plain strip: S tiles at once; the row strip of tile (I,K) is staged once in
// shared memory and serves the S columns of every lane.
template <int S>
__device__ __forceinline__ void far_strip_plain(const FoldParams &P, const SeqDesc &sd, int I, int J0, int Seff, int Ka,
                                                int Kb, unsigned (&acc)[S][32], WarpScratch<8, kPlain> &ws, int lane) {
    constexpr int T = 32;
    const int Np = sd.Np, PC = sd.PC;
    const int16_t *Drow = P.drow + sd.drow_off;
    const int16_t *Dcol = P.dcol + sd.dcol_off;
    uint4 rown[4];
    uint4 coln[S][4];
    auto load = [&](int K) {
        const uint4 *src = reinterpret_cast<const uint4 *>(Drow + (size_t)(I * T + lane) * Np + K * T);
#pragma unroll
        for (int v = 0; v < 4; ++v) rown[v] = __ldcg(src + v);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint4 *cs = reinterpret_cast<const uint4 *>(Dcol + (size_t)((J0 + s) * T + lane) * PC + K * T + 1 + kColOff);
#pragma unroll
            for (int v = 0; v < 4; ++v) coln[s][v] = (s < Seff) ? __ldcg(cs + v) : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    load(Ka);
    for (int K = Ka; K <= Kb; ++K) {
        unsigned col[S][16];
        uint4 *dst = reinterpret_cast<uint4 *>(&ws.rows[lane][0]);
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = rown[v];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                col[s][4 * v] = coln[s][v].x; col[s][4 * v + 1] = coln[s][v].y;
                col[s][4 * v + 2] = coln[s][v].z; col[s][4 * v + 3] = coln[s][v].w;
            }
        if (K < Kb) load(K + 1);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < T; ++r) {
            const uint4 *rw = reinterpret_cast<const uint4 *>(&ws.rows[r][0]);
            const uint4 a0 = rw[0], a1 = rw[1], a2 = rw[2], a3 = rw[3];
            const unsigned aw[16] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w,
                                     a2.x, a2.y, a2.z, a2.w, a3.x, a3.y, a3.z, a3.w};
#pragma unroll
            for (int s = 0; s < S; ++s) {
                unsigned x = acc[s][r];
#pragma unroll
                for (int w = 0; w < 16; ++w) x = __viaddmax_s16x2(aw[w], col[s][w], x);
                acc[s][r] = x;
            }
        }
        __syncwarp();
    }
}

// A strip's partial maxima merged by bulk reductions: each tile's values (value(s2, r) for column
// lane, row r) are staged in pbuf (free once the lookups are done: it shares its bytes with the chunk
// staging) and reduced into the tile's P slot by one bulk operation; the next tile is staged once
// the previous source has been read.  Lane 0 then waits for every reduction, fences the async
// proxy's writes and publishes the tiles' counts.
template <int Q, int M, int S, class V>
__device__ __forceinline__ void merge_strip_bulk(const FoldParams &P, const SeqDesc &sd, int I, int J0, int Seff,
                                                 WarpScratch<Q, M> &ws, int lane, NextTask &nt, V value) {
    constexpr int T = Cfg<Q, M>::T;
    const int NT = sd.NT;
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
        if (s2 >= Seff) continue;
        if (s2 > 0 && lane == 0) bulk_wait_read_all();
        __syncwarp();
        if (lane < T) {
#pragma unroll
            for (int r = 0; r < T; ++r) ws.pbuf[r * T + lane] = value(s2, r);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            int *slot = P.pring + sd.p_off + ((size_t)((J0 + s2 - I) % kRing) * NT + I) * (T * T);
            // the slot's earlier zeroing (generic proxy, acquired with the input flags) before the
            // async proxy's reduction into it
            if (s2 == 0) fence_proxy_async_global();
            bulk_red_max_s32(slot, ws.pbuf, (unsigned)(T * T * sizeof(int)));
            bulk_commit();
        }
    }
    nt.finish(lane);
    if (lane == 0) {
        bulk_wait_all();
        fence_proxy_async_global();
        fence_acq_rel();   // releases the merges with the relaxed counts below
        for (int s2 = 0; s2 < Seff; ++s2) red_add(P.cnt + sd.cnt_off + I * NT + J0 + s2, 1);
    }
    __syncwarp();
}

template <int Q, int M, bool MEMO>
__device__ __forceinline__ long long run_far_strip(const FoldParams &P, const SeqDesc &sd, int I, int J0, int Ka,
                                                   int Kb, WarpScratch<Q, M> &ws, const uint8_t *Rs, int lane,
                                                   long long *tdeps, NextTask &nt) {
    constexpr int T = Cfg<Q, M>::T;
    constexpr int S = strip_of(Q, M);
    const int NT = sd.NT;
    int *flags = P.flags + sd.flag_off;
    const int Seff = min(S, NT - J0);
    const int Jl = J0 + Seff - 1;
    if (Seff < 1 || Kb < Ka || Ka < I + 2 || Kb > J0 - 2) {
        if (lane == 0) atomicCAS(P.error, 0, kErrBadTask);
        return 0;
    }
    if (!warp_wait_flags(flags + I * NT + Kb, flags + Ka * NT + Jl,
                         Jl - I >= kRing ? flags + I * NT + (Jl - kRing) : nullptr, P, lane))
        return 0;
    if (P.trace) tdeps[0] = (long long)gtimer();
    long long tdone = 0;
    if constexpr (M == kTwoVector) {
        unsigned m2[S / 2][T];
#pragma unroll
        for (int p2 = 0; p2 < S / 2; ++p2)
#pragma unroll
            for (int r = 0; r < T; ++r) m2[p2][r] = 0u;
        far_strip_tv<Q, S, MEMO>(P, sd, I, J0, Seff, Ka, Kb, m2, ws, Rs, lane);
        if (P.trace) tdone = (long long)gtimer();
        nt.start(lane);
        if constexpr (WarpScratch<Q, M>::PB) {
            merge_strip_bulk<Q, M, S>(P, sd, I, J0, Seff, ws, lane, nt, [&](int s2, int r) {
                return (s2 & 1) ? (int)(m2[s2 / 2][r] >> 16) : (int)(m2[s2 / 2][r] & 0xffffu);
            });
            return tdone;
        }
        if (lane < T) {
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) {
                if (s2 >= Seff) continue;
                int *slot = P.pring + sd.p_off + ((size_t)((J0 + s2 - I) % kRing) * NT + I) * (T * T);
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    const int v = (s2 & 1) ? (int)(m2[s2 / 2][r] >> 16) : (int)(m2[s2 / 2][r] & 0xffffu);
                    if (v > 0) red_max(slot + r * T + lane, v);
                }
            }
        }
    } else {
        unsigned acc[S][32];
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2)
#pragma unroll
            for (int r = 0; r < 32; ++r) acc[s2][r] = 0u;
        far_strip_plain<S>(P, sd, I, J0, Seff, Ka, Kb, acc, ws, lane);
        if (P.trace) tdone = (long long)gtimer();
        nt.start(lane);
        if constexpr (WarpScratch<Q, M>::PB) {
            merge_strip_bulk<Q, M, S>(P, sd, I, J0, Seff, ws, lane, nt,
                                      [&](int s2, int r) { return hmax2(acc[s2][r]); });
            return tdone;
        }
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
            if (s2 >= Seff) continue;
            int *slot = P.pring + sd.p_off + ((size_t)((J0 + s2 - I) % kRing) * NT + I) * (T * T);
#pragma unroll
            for (int r = 0; r < T; ++r) {
                const int v = hmax2(acc[s2][r]);
                if (v > 0) red_max(slot + r * T + lane, v);
            }
        }
    }
    nt.finish(lane);
    __threadfence();
    __syncwarp();
    if (lane < Seff) atomicAdd(P.cnt + sd.cnt_off + I * NT + J0 + lane, 1);
    return tdone;
}

// ---------------------------------------------------------------- NEAR task
// Column mode: what the warp owning tile column J carries from tile (I+1,J) to tile (I,J), and the
// link to the warp of column J-1 when that warp runs in the same CTA.
template <int Q, int M>
struct NearCol {
    static constexpr int G = Cfg<Q, M>::G;
    int k;                        // index of the tile in the column: tile (J-k, J), t = k
    WarpScratch<Q, M> *prod;      // scratch of the warp of column J-1 in this CTA, or null
    bool consumer;                // the warp of column J+1 runs in this CTA and reads this warp's tiles
    unsigned Wp[16];              // W[c'][c] of tile (J,J), packed pairs (set by tile 0)
    uint32_t lcb0[G];             // two-vector: features (B << 16 | c) of middle block J-1 in column j (set by tile 1)
    unsigned lcol0[16];           // plain: column j of tile (J-1,J), packed pairs (set by tile 1)
    int colT;                     // D(IT, j) of the tile just finished: row 0 of the next tile's bottom neighbour
    bool cnt_ok;                  // the next tile's chunk counter was complete when the last tile released
    const int4 *tasks;            // tile tasks in diagonal order (chunk counts)
    bool failed;                  // the last tile stopped on a failed wait
};

template <int Q, int M, bool COL, bool MEMO>
__device__ __forceinline__ long long run_near(const FoldParams &P, const SeqDesc &sd, int I, int J, int nfar,
                                              WarpScratch<Q, M> &ws, const uint8_t *Rs, int lane, long long *tdeps,
                                              NearCol<Q, M> &cs) {
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
    const uint32_t *RF = P.rf + sd.rf_off;
    const uint32_t *CF = P.cf + sd.cf_off;
    const int NG = TV ? Np / Q : 1;
    const bool lateA = t >= 2;   // middle block K = J-1: rows of tile (I,J-1) x column of tile (J-1,J)
    const bool lateB = t >= 3;   // middle block K = I+1: rows of tile (I,I+1) x column of tile (I+1,J)
    // column mode: tiles alternate between two buffers; the previous one holds tile (I+1,J)
    const int buf = COL ? (cs.k & 1) : 0;
    int16_t(*tile)[33] = buf ? ws.tile1 : ws.tile;
    const int16_t(*ptile)[33] = buf ? ws.tile : ws.tile1;
    WarpScratch<Q, M> *prod = COL ? cs.prod : nullptr;
    const int pbp = (cs.k - 1) & 1;   // buffer of the producer's tile (I, J-1)
    // old-tile inputs: diagonal tile rows and features, late block K = I+1 rows
    auto &dg = ws.diag;
    auto &lrf1 = ws.lrf[1];
    auto &lrow1 = ws.lrow[1];
    if constexpr (COL) cs.failed = true;   // cleared when the tile completes
    // column mode, chunk counter already seen complete: no wait, and the loads of old tiles go out
    // before the left neighbour is awaited
    const bool early = COL && nfar > 0 && cs.cnt_ok;
    int acc[T];
    int *slot = P.pring + sd.p_off + ((size_t)(t % kRing) * NT + I) * (T * T);
    // codes of the tile's rows (one per lane) and of this lane's column, for the pair bits
    const int rcode = lane < T ? (int)codes[IT + lane] : kPadCode;
    const int sj = valid ? (int)codes[j] : kPadCode;
    // column mode: chunk count of the column's next tile (I-1, J)
    const int nn_next = (COL && I > 0) ? __ldg(&cs.tasks[(t + 1) * NT - (t + 1) * t / 2 + (I - 1)].z) : 0;

    // ---- inputs from tiles finished long before the neighbours, all loads in flight at once
    unsigned Wp[16];           // packed W[c'][c] = D(JT+c'+1, j) for c' < c, 0 for c' = c (the empty
                               // interval: the closure then carries the column's own pair term),
                               // sentinel otherwise
    uint32_t lcb[2][G];        // late-block column features (B << 16 | c) (two-vector)
    unsigned lcol[2][16];      // late-block columns as packed pairs (plain)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
        for (int gl = 0; gl < G; ++gl) lcb[k][gl] = 0u;
#pragma unroll
        for (int v = 0; v < 16; ++v) lcol[k][v] = 0;
    }
    // column mode: the tile's P slot goes to shared memory by cp.async, at once when its chunk counter
    // was already seen complete (the copy then overlaps the wait for the left neighbour)
    constexpr bool PBC = COL && WarpScratch<Q, M>::PB;
    auto p_copy = [&]() {
        if constexpr (PBC) {
            const int4 *src = reinterpret_cast<const int4 *>(slot);
            int4 *dst = reinterpret_cast<int4 *>(ws.pbuf);
#pragma unroll
            for (int k = lane; k < T * T / 4; k += 32) cp_async16(dst + k, src + k);
            cp_async_commit();
        }
    };
    if constexpr (COL) {
        // the next column's warp must have read the tile two back before its buffer is rewritten
        if (cs.consumer && cs.k >= 2 && !wait_smem_geq(&ws.consumed, cs.k - 1, P.error, P.timeout_ns, lane)) return 0;
        if (early) p_copy();
        // left neighbour (I, J-1), from the warp of column J-1 in this CTA or else through its flag; it
        // implies every tile of row I to its left, (I,I) and (I,I+1) among them.  The bottom neighbour
        // (I+1, J) is this warp's previous tile.  A complete chunk counter (seen before the last
        // release) implies them too: the chunk of middle block I+2 waited for tile (I, I+2).  Then the
        // loads of old tiles go out first and the left neighbour is awaited after them.
        if (t >= 1 && !early) {
            if (prod) {
                if (!wait_smem_geq(&prod->produced, cs.k, P.error, P.timeout_ns, lane)) return 0;
            } else if (!warp_wait_geq(flags + I * NT + (J - 1), 1, P, lane)) {
                return 0;
            }
        }
    }
    // the flags a tile reads (not column mode): 0-3 old tiles (I,I), (J,J), (J-1,J) and (I,I+1) for
    // the late blocks, 4-5 the neighbours (I,J-1) and (I+1,J); null = not read
    auto flag_ptr = [&](int k) -> const int * {
        return k == 0 ? flags + I * NT + I
             : k == 1 ? flags + J * NT + J
             : k == 2 ? (lateA ? flags + (J - 1) * NT + J : nullptr)
             : k == 3 ? (lateB ? flags + I * NT + (I + 1) : nullptr)
             : k == 4 ? flags + I * NT + (J - 1)
             : k == 5 ? flags + (I + 1) * NT + J : nullptr;
    };
    unsigned nb_miss = 0;      // neighbour flags not seen set yet (bits 4 and 5)
    if (t >= 1) {
        if constexpr (!COL) {
            // lanes 0-5 acquire one flag each, so the usual case (all set) costs one round trip; the
            // warp barrier orders every lane's later loads after the acquires (as in wait_geq_impl).
            // An old tile not yet done is awaited now, a neighbour after the old tiles' loads.
            const int *mine = flag_ptr(lane);
            const unsigned miss = __ballot_sync(FULL, mine != nullptr && ld_acquire(mine) < 1);
            __syncwarp();
            for (unsigned m = miss & 0xfu; m; m &= m - 1)
                if (!warp_wait_geq(flag_ptr(__ffs(m) - 1), 1, P, lane)) return 0;
            nb_miss = miss & 0x30u;
        }
        int16_t dv[T];
#pragma unroll
        for (int r = 0; r < T; ++r)
            dv[r] = valid ? __ldcg(Drow + (size_t)(IT + r) * Np + IT + c) : (int16_t)0;
        if constexpr (COL) {
#pragma unroll
            for (int mm = 0; mm < 16; ++mm) Wp[mm] = cs.Wp[mm];
        } else {
#pragma unroll
            for (int mm = 0; mm < 16; ++mm) {
                const int c0 = 2 * mm, c1 = 2 * mm + 1;
                int w0 = (valid && c0 == c) ? 0 : kNeg16, w1 = (valid && c1 == c) ? 0 : kNeg16;
                // D(JT+c'+1, j): two-vector from the row-major table (one 64-byte row segment per
                // load: batch kernel -6%); the plain kernel measured faster with its column copy
                if constexpr (TV) {
                    if (valid && c0 < c) w0 = ldcg16(Drow + (size_t)(JT + c0 + 1) * Np + j);
                    if (valid && c1 < c) w1 = ldcg16(Drow + (size_t)(JT + c1 + 1) * Np + j);
                } else {
                    if (valid && c0 < c) w0 = ldcg16(Dcol + (size_t)j * PC + JT + c0 + 1 + kColOff);
                    if (valid && c1 < c) w1 = ldcg16(Dcol + (size_t)j * PC + JT + c1 + 1 + kColOff);
                }
                Wp[mm] = (unsigned)(w0 & 0xffff) | ((unsigned)w1 << 16);
            }
        }
        if constexpr (TV) {
            constexpr int E = (T * G + 31) / 32;   // row features of (I,I) and (I,I+1), spread over the warp
            uint32_t fv[E], fb[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = e * 32 + lane;
                const bool in = idx < T * G;
                const size_t row = (size_t)(IT + idx / G) * NG;
                fv[e] = in ? __ldcg(RF + row + I * G + idx % G) : 0u;
                fb[e] = (in && lateB) ? __ldcg(RF + row + (I + 1) * G + idx % G) : 0u;
            }
            if (lateA && valid) {
#pragma unroll
                for (int gl = 0; gl < G; ++gl) {
                    if constexpr (COL) {
                        lcb[0][gl] = cs.lcb0[gl];
                    } else {
                        const uint32_t cf = __ldcg(CF + (size_t)((J - 1) * G + gl) * Np + j);
                        lcb[0][gl] = cf;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = e * 32 + lane;
                memo_ensure<Q, M, MEMO>(Rs, fv[e] & C::BMASK, idx < T * G, lane);
                memo_ensure<Q, M, MEMO>(Rs, fb[e] & C::BMASK, idx < T * G && lateB, lane);
                if (idx < T * G) {
                    // the row's word for group gl: A, or -32768 while the group is not complete
                    // below the row (gl*q <= row), and the R-row offset of h
                    const int rw = idx / G, gl = idx % G;
                    const uint32_t hw = C::NIB ? (fv[e] & C::BMASK) : (uint32_t)hrow_offset<Q>((int)(fv[e] & C::BMASK));
                    const uint32_t aw = (gl * Q > rw) ? (fv[e] & 0xffff0000u) : 0x80000000u;
                    ws.gw[rw][gl] = aw | hw;
                    lrf1[rw][gl] = group_word<Q>(fb[e]);
                }
            }
        } else {
            if (lateB) {   // row strip of tile (I, I+1), row IT+lane
                const uint4 *src = reinterpret_cast<const uint4 *>(Drow + (size_t)(IT + lane) * Np + (I + 1) * T);
                uint4 *dst = reinterpret_cast<uint4 *>(&lrow1[lane][0]);
#pragma unroll
                for (int v = 0; v < 4; ++v) dst[v] = __ldcg(src + v);
            }
            if (lateA) {   // column j of tile (J-1, J): rows (J-1)T+1 .. JT
                if constexpr (COL) {
#pragma unroll
                    for (int v = 0; v < 16; ++v) lcol[0][v] = cs.lcol0[v];
                } else {
                    const uint4 *cp = reinterpret_cast<const uint4 *>(Dcol + (size_t)j * PC + (J - 1) * T + 1 + kColOff);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        uint4 w = __ldcg(cp + v);
                        lcol[0][4 * v] = w.x; lcol[0][4 * v + 1] = w.y; lcol[0][4 * v + 2] = w.z; lcol[0][4 * v + 3] = w.w;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < T; ++r)
            if (valid) dg[r][c] = dv[r];
    } else {
#pragma unroll
        for (int mm = 0; mm < 16; ++mm) Wp[mm] = 0;
    }

    // ---- the two neighbours that finish last
    if constexpr (!COL) {
        for (unsigned m = nb_miss; m; m &= m - 1)
            if (!warp_wait_geq(flag_ptr(__ffs(m) - 1), 1, P, lane)) return 0;
    } else {
        if (t >= 1 && early) {
            const bool ok = prod ? wait_smem_geq(&prod->produced, cs.k, P.error, P.timeout_ns, lane)
                                 : warp_wait_geq(flags + I * NT + (J - 1), 1, P, lane);
            if (!ok) {
                if constexpr (PBC) cp_async_wait_all();   // no copy is left in flight
                return 0;
            }
        }
    }
    if (P.trace) tdeps[0] = (long long)gtimer();
    // every load that depends on the neighbours goes out at once
    int colT = 0;              // D((I+1)T, j): row 0 of tile (I+1, J)
    int leftv = 0;             // D(IT+1+c, JT-1): left column for lane 0's pair term
    if (t >= 1 && valid) {
        const int row = IT + 1 + c;
        if constexpr (COL) {
            colT = cs.colT;
            if (prod) {
                // the producer's tile has row T = D((I+1)T, JT-1), which is 0 when t = 1
                const int16_t(*pt)[33] = pbp ? prod->tile1 : prod->tile;
                leftv = (int)pt[c + 1][T - 1];
            } else if (row <= JT - 1 && row < Np) {
                // two-vector column mode keeps no column-major copy
                leftv = TV ? ldcg16(Drow + (size_t)row * Np + (JT - 1)) : ldcg16(Dcol + (size_t)(JT - 1) * PC + row + kColOff);
            }
        } else {
            if ((I + 1) * T < Np) colT = ldcg16(Drow + (size_t)((I + 1) * T) * Np + j);
            if (row <= JT - 1 && row < Np) leftv = ldcg16(Dcol + (size_t)(JT - 1) * PC + row + kColOff);
        }
    }
    constexpr int E = (T * G + 31) / 32;
    uint32_t fa[E];            // row features of tile (I, J-1) (two-vector, late block K = J-1)
    uint4 ra[4];               // row strip of tile (I, J-1), row IT+lane (plain)
    if constexpr (TV) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = e * 32 + lane;
            const bool in = lateA && idx < T * G;
            if (COL && prod) fa[e] = in ? prod->rfo[pbp][idx / G][idx % G] : 0u;
            else fa[e] = in ? __ldcg(RF + (size_t)(IT + idx / G) * NG + (J - 1) * G + idx % G) : 0u;
        }
        if (lateB && valid) {
#pragma unroll
            for (int gl = 0; gl < G; ++gl) {
                // column mode: the features of block I+1 are this warp's previous tile's
                const uint32_t cf = COL ? ws.cbc[c][gl] : __ldcg(CF + (size_t)((I + 1) * G + gl) * Np + j);
                lcb[1][gl] = cf;
            }
        }
        // this tile's column groups start as (B, c) = (0, 0): a group that is not complete below a
        // row then adds at most -32768 + q - 1 there (its A is -32768)
#pragma unroll
        for (int g4 = 0; g4 < WarpScratch<Q, M>::GA / 4; ++g4)
            reinterpret_cast<uint4 *>(&ws.cbc[c][0])[g4] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        if (COL && prod) {
            const int16_t(*pt)[33] = pbp ? prod->tile1 : prod->tile;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                unsigned w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = lateA ? ((unsigned)(uint16_t)pt[lane][8 * v + 2 * e] | ((unsigned)(uint16_t)pt[lane][8 * v + 2 * e + 1] << 16)) : 0u;
                ra[v] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        } else {
            const uint4 *src = reinterpret_cast<const uint4 *>(Drow + (size_t)(IT + lane) * Np + (J - 1) * T);
#pragma unroll
            for (int v = 0; v < 4; ++v) ra[v] = lateA ? __ldcg(src + v) : make_uint4(0u, 0u, 0u, 0u);
        }
        if (lateB) {   // column j of tile (I+1, J): rows (I+1)T+1 .. (I+2)T
            if constexpr (COL) {
#pragma unroll
                for (int w = 0; w < 16; ++w)
                    lcol[1][w] = (unsigned)(uint16_t)ptile[1 + 2 * w][c] | ((unsigned)(uint16_t)ptile[2 + 2 * w][c] << 16);
            } else {
                const uint4 *cp = reinterpret_cast<const uint4 *>(Dcol + (size_t)j * PC + (I + 1) * T + 1 + kColOff);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    uint4 w = __ldcg(cp + v);
                    lcol[1][4 * v] = w.x; lcol[1][4 * v + 1] = w.y; lcol[1][4 * v + 2] = w.z; lcol[1][4 * v + 3] = w.w;
                }
            }
        }
    }
    if constexpr (COL) {
        // everything of the producer's tile has been read: its buffer may be reused
        if (prod && t >= 1) {
            __syncwarp();
            if (lane == 0) st_release_cta(&prod->consumed, cs.k);
        }
    }
    // partial max of the FAR chunks (middle blocks I+2 .. J-2)
    if (nfar > 0) {
        if (!early && !warp_wait_geq(P.cnt + sd.cnt_off + I * NT + J, nfar, P, lane)) return 0;
        if constexpr (PBC) {
            if (!early) p_copy();
            cp_async_wait_all();
            __syncwarp();
#pragma unroll
            for (int r = 0; r < T; ++r) acc[r] = valid ? ws.pbuf[r * T + c] : 0;
        } else {
#pragma unroll
            for (int r = 0; r < T; ++r) acc[r] = valid ? __ldcg(slot + r * T + c) : 0;
        }
        if (P.trace) tdeps[1] = (long long)gtimer();
    } else {
#pragma unroll
        for (int r = 0; r < T; ++r) acc[r] = 0;
    }
    if constexpr (TV) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = e * 32 + lane;
            memo_ensure<Q, M, MEMO>(Rs, fa[e] & C::BMASK, idx < T * G && lateA, lane);
            if (idx < T * G) ws.lrf[0][idx / G][idx % G] = group_word<Q>(fa[e]);
        }
    } else {
        uint4 *dst = reinterpret_cast<uint4 *>(&ws.lrow[0][lane][0]);
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = ra[v];
    }
    __syncwarp();
    if constexpr (TV) {
        // per row of the diagonal tile (lane = row), the residual splits' D(i, k-1) in int16 pairs:
        // slot e holds k = i+2+e while k is at most the end ce of the first group that starts after
        // the row, -32768 otherwise (the groups from ce on are full groups of the row)
        using WS = WarpScratch<Q, M>;
        if (t >= 1 && lane < T) {
            const int rr = lane;
            const int ce = (rr / Q + 1) * Q;
            uint32_t w[WS::NWPA];
#pragma unroll
            for (int k = 0; k < WS::NWPA; ++k) w[k] = 0x80008000u;
#pragma unroll
            for (int e = 0; e < NW_RES<Q>; ++e) {
                const int kk = rr + 2 + e;
                const uint32_t v = (kk <= ce) ? (uint32_t)(uint16_t)dg[rr][min(kk, T) - 1] : 0x8000u;
                w[e >> 1] = (e & 1) ? ((w[e >> 1] & 0xffffu) | (v << 16)) : ((w[e >> 1] & 0xffff0000u) | v);
            }
#pragma unroll
            for (int k4 = 0; k4 < WS::NWPA / 4; ++k4)
                reinterpret_cast<uint4 *>(&ws.rpk[rr][0])[k4] = make_uint4(w[4 * k4], w[4 * k4 + 1], w[4 * k4 + 2], w[4 * k4 + 3]);
        }
    }
    // the two late middle blocks for every row at once (independent lookups, high ILP)
    if constexpr (TV) {
        // acc is scaled by 2^16 while the group terms are merged (see group_term)
#pragma unroll
        for (int r = 0; r < T; ++r) acc[r] = (int)((unsigned)acc[r] << 16);
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
            if (kb == 0 ? lateA : lateB) {
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    uint32_t fr[G];   // the row's features, one 16-byte load per four groups
                    if constexpr (G % 4 == 0) {
                        const uint4 *pv = reinterpret_cast<const uint4 *>(kb == 0 ? &ws.lrf[0][r][0] : &lrf1[r][0]);
#pragma unroll
                        for (int v4 = 0; v4 < G / 4; ++v4) {
                            const uint4 w = pv[v4];
                            fr[4 * v4] = w.x; fr[4 * v4 + 1] = w.y; fr[4 * v4 + 2] = w.z; fr[4 * v4 + 3] = w.w;
                        }
                    } else {
#pragma unroll
                        for (int gl = 0; gl < G; ++gl) fr[gl] = kb == 0 ? ws.lrf[0][r][gl] : lrf1[r][gl];
                    }
#pragma unroll
                    for (int gl = 0; gl < G; ++gl) acc[r] = max(acc[r], group_term<Q>(Rs, fr[gl], lcb[kb][gl]));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < T; ++r) acc[r] >>= 16;
    } else {
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
            if (kb == 0 ? lateA : lateB) {
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    const uint4 *rw = reinterpret_cast<const uint4 *>(kb == 0 ? &ws.lrow[0][r][0] : &lrow1[r][0]);
                    unsigned a0 = 0, a1 = 0;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const uint4 a = rw[v];
                        a0 = __viaddmax_s16x2(a.x, lcol[kb][4 * v + 0], a0);
                        a1 = __viaddmax_s16x2(a.y, lcol[kb][4 * v + 1], a1);
                        a0 = __viaddmax_s16x2(a.z, lcol[kb][4 * v + 2], a0);
                        a1 = __viaddmax_s16x2(a.w, lcol[kb][4 * v + 3], a1);
                    }
                    acc[r] = max(acc[r], hmax2(__vmaxs2(a0, a1)));
                }
            }
        }
    }
    if (valid) {
#pragma unroll
        for (int r = 0; r < T; ++r) ws.pm[r][c] = (int16_t)acc[r];
    }
    if (nfar > 0 && J + kRing < NT) {   // ring slot reused by tile (I, J+kRing)
        if constexpr (PBC) {
#pragma unroll
            for (int k = lane; k < T * T / 4; k += 32) __stcg(reinterpret_cast<int4 *>(slot) + k, make_int4(0, 0, 0, 0));
        } else if (valid) {
#pragma unroll
            for (int r = 0; r < T; ++r) __stcg(slot + r * T + c, 0);
        }
    }
    const long long tfar = P.trace ? (long long)gtimer() : 0;

    if (valid) {
        ws.left[c + 1] = (int16_t)leftv;
        tile[T][c] = (int16_t)colT;
    }
    if (c == 0) ws.left[0] = 0;
    if constexpr (!TV) {
        // column pairs (D(IT+2m+1,j), D(IT+2m+2,j)); rows not yet computed hold the sentinel
#pragma unroll
        for (int mm = 0; mm < 16; ++mm)
            ws.colpk[mm][c] = (mm == 15) ? ((unsigned)(kNeg16 & 0xffff) | ((unsigned)colT << 16))
                                         : ((unsigned)(kNeg16 & 0xffff) | ((unsigned)(kNeg16 & 0xffff) << 16));
    }
    __syncwarp();

    unsigned vhist = 0;        // vertical differences, newest in bit 0
    // residual window (two-vector), int16 pairs: value e = D(IT+r+1+e, j) while row r is being
    // computed, in half e&1 of wpk[e/2]
    using WS = WarpScratch<Q, M>;
    unsigned wpk[WS::NWP];
#pragma unroll
    for (int e = 0; e < WS::NWP; ++e) wpk[e] = 0u;
    wpk[0] = (unsigned)colT & 0xffffu;

    // terms of row rr that do not depend on row rr+1 (computed while row rr+1 closes); branch-free:
    // every candidate is evaluated with in-range indices and the invalid ones are masked
    auto old_terms = [&](int rr) -> int {
        if constexpr (TV) {
            int best = (int)ws.pm[rr][c];
            // residual splits k in [i+2, IT+ce], ce the end of the first group starting after row rr
            // (k = i+1 is the D(i+1,j) term of the row loop); on a group's first row they cover that
            // whole group, so no term of a row waits on the group its previous row completes
            unsigned ra = 0u, rb = 0u;
#pragma unroll
            for (int k4 = 0; k4 < WS::NWPA / 4; ++k4) {
                const uint4 a = reinterpret_cast<const uint4 *>(&ws.rpk[rr][0])[k4];
                if (4 * k4 + 0 < WS::NWP) ra = __viaddmax_s16x2(a.x, wpk[min(4 * k4 + 0, WS::NWP - 1)], ra);
                if (4 * k4 + 1 < WS::NWP) rb = __viaddmax_s16x2(a.y, wpk[min(4 * k4 + 1, WS::NWP - 1)], rb);
                if (4 * k4 + 2 < WS::NWP) ra = __viaddmax_s16x2(a.z, wpk[min(4 * k4 + 2, WS::NWP - 1)], ra);
                if (4 * k4 + 3 < WS::NWP) rb = __viaddmax_s16x2(a.w, wpk[min(4 * k4 + 3, WS::NWP - 1)], rb);
            }
            best = max(best, hmax2(__vmaxs2(ra, rb)));
            // full groups of tile column I after that one (g*q > rr; the others carry A = -32768),
            // complete before row rr+1
            int gm = (int)0x80000000u;
#pragma unroll
            for (int g4 = 0; g4 < WS::GA / 4; ++g4) {
                const uint4 gv = reinterpret_cast<const uint4 *>(&ws.gw[rr][0])[g4];
                const uint4 cv = reinterpret_cast<const uint4 *>(&ws.cbc[c][0])[g4];
                if (4 * g4 + 0 < G) gm = max(gm, group_term<Q>(Rs, gv.x, cv.x));
                if (4 * g4 + 1 < G) gm = max(gm, group_term<Q>(Rs, gv.y, cv.y));
                if (4 * g4 + 2 < G) gm = max(gm, group_term<Q>(Rs, gv.z, cv.z));
                if (4 * g4 + 3 < G) gm = max(gm, group_term<Q>(Rs, gv.w, cv.w));
            }
            return max(best, gm >> 16);
        } else {
            // every split with D(k,j) in this tile column: rows not yet done hold the sentinel
            unsigned acc2[4] = {0u, 0u, 0u, 0u};
            const uint4 *dw = reinterpret_cast<const uint4 *>(&dg[rr][0]);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint4 a = dw[v];
                acc2[0] = __viaddmax_s16x2(a.x, ws.colpk[4 * v + 0][c], acc2[0]);
                acc2[1] = __viaddmax_s16x2(a.y, ws.colpk[4 * v + 1][c], acc2[1]);
                acc2[2] = __viaddmax_s16x2(a.z, ws.colpk[4 * v + 2][c], acc2[2]);
                acc2[3] = __viaddmax_s16x2(a.w, ws.colpk[4 * v + 3][c], acc2[3]);
            }
            const unsigned m2 = __vmaxs2(__vmaxs2(acc2[0], acc2[1]), __vmaxs2(acc2[2], acc2[3]));
            return max((int)ws.pm[rr][c], hmax2(m2));
        }
    };

    // publishes row r (value d of this lane's column): tile copy, row-major store, vertical and
    // horizontal difference vectors
    auto publish = [&](int r, int d, int below_prev) {
        tile[r][c] = (int16_t)d;
        if (T == 32 || valid) Drow[(size_t)(IT + r) * Np + j] = (int16_t)d;
        const int vb = d - below_prev;   // vertical difference D(i,j) - D(i+1,j)
        vhist = (vhist << 1) | (unsigned)(vb & 1);
        if constexpr (TV) {
            const bool done = r >= 1 && (r - 1) % Q == 0;   // group rows gl*q+1 .. gl*q+q complete
            const int gl = max(r - 1, 0) / Q;
            const uint32_t cb = ((uint32_t)d << 16) | (vhist & C::BMASK);
            if (done) ws.cbc[c][gl] = cb;
            if (done && valid) P.cf[sd.cf_off + (size_t)(I * G + gl) * Np + j] = cb;
        } else {
            // row r joins the column pairs used by the rows above
            const int mm = max(r - 1, 0) >> 1;
            const uint32_t w = ws.colpk[mm][c];
            const uint32_t w2 = (r & 1) ? ((w & 0xffff0000u) | ((uint32_t)d & 0xffffu)) : ((w & 0xffffu) | ((uint32_t)d << 16));
            ws.colpk[mm][c] = (r >= 1) ? w2 : w;
        }
    };

    // pair bits of this lane's column against the tile's rows, bit r = b(S_{IT+r}, S_j): one ballot
    // per base the column may hold (padding codes pair with nothing)
    unsigned pbits;
    {
        unsigned pbx[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) pbx[x] = __ballot_sync(FULL, (P.pair64 >> (8 * rcode + x)) & 1ull);
        pbits = sj == 0 ? pbx[0] : sj == 1 ? pbx[1] : sj == 2 ? pbx[2] : sj == 3 ? pbx[3] : 0u;
    }
    int below = colT;          // D(i+1, j)
    if (t == 0) {
        // diagonal tile: every split lies in this tile, so the closure alone covers them; W is this
        // tile's own column D(IT+c'+1, j), valid for r <= c' < c
#pragma unroll 1
        for (int r = T - 1; r >= 0; --r) {
            const int pb = (int)((pbits >> r) & 1u);
            const int blraw = __shfl_up_sync(FULL, below, 1);
            const int bl = (c == 0) ? 0 : blraw;
            int y = (c > r) ? pb + bl : (c == r ? 0 : kNeg16);
            y = valid ? y : kNeg16;
            ws.y[r & 1][c] = (int16_t)y;
            __syncwarp();
            const uint4 *yp = reinterpret_cast<const uint4 *>(ws.y[r & 1]);
            unsigned a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint4 a = yp[v];
                const unsigned aw[4] = {a.x, a.y, a.z, a.w};
                unsigned wp[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c0 = 8 * v + 2 * e, c1 = c0 + 1;
                    const int r0 = (c0 + 1 <= T) ? c0 + 1 : T, r1 = (c1 + 1 <= T) ? c1 + 1 : T;
                    const int t0 = (int)tile[r0][c], t1 = (int)tile[r1][c];
                    const int w0 = (c0 < c && c0 >= r && c0 + 1 <= T) ? t0 : kNeg16;
                    const int w1 = (c1 < c && c1 >= r && c1 + 1 <= T) ? t1 : kNeg16;
                    wp[e] = (unsigned)(w0 & 0xffff) | ((unsigned)w1 << 16);
                }
                a0 = __viaddmax_s16x2(aw[0], wp[0], a0);
                a1 = __viaddmax_s16x2(aw[1], wp[1], a1);
                a2 = __viaddmax_s16x2(aw[2], wp[2], a2);
                a3 = __viaddmax_s16x2(aw[3], wp[3], a3);
            }
            const unsigned acc = __vmaxs2(__vmaxs2(a0, a1), __vmaxs2(a2, a3));
            int d = max(y, hmax2(acc));
            d = (c < r || !valid) ? 0 : d;
            publish(r, d, below);
            below = d;
        }
    } else {
        int yold = old_terms(T - 1);
        // closure over the row, D_c = max(Y_c, max_{c'<=c} Y'_c' + W[c'][c]).  Only the pair term of
        // Y_c' can matter there: every other term of Y_c' is a split D(i,k-1) + D(k,JT+c'), and with
        // W[c'][c] added it is at most D(i,k-1) + D(k,j) (superadditivity, Eq. 1), a term Y_c or the
        // closure already holds.  So the exchanged value is Y'_c' = D(i+1, JT+c'-1) + b(S_i, S_{JT+c'})
        // (W[c][c] = 0 brings in the column's own pair term); where b = 0 it is the split of
        // D(i+1, j) = below into two disjoint parts, at most that and harmless.  Y' needs no select:
        // lane c'-1 stores its own value of the row below plus column c''s pair bit at position c' of
        // ws.y right after it computes it, and lane 31 stores the left column's value at position 0.
        const unsigned pbn = __shfl_sync(FULL, pbits, (lane + 1) & 31);   // column c+1's pair bits
        const int yslot = (c + 1) & 31;
        {
            const int bv = c == 31 ? (int)ws.left[T] : colT;
            ws.y[(T - 1) & 1][yslot] = (int16_t)(bv + (int)((pbn >> (T - 1)) & 1u));
        }
        __syncwarp();
#pragma unroll 2
        for (int r = T - 1; r >= 0; --r) {
            // the closure's inputs go out first; the work below fills their latency
            const uint4 *yp = reinterpret_cast<const uint4 *>(ws.y[r & 1]);
            uint4 ya[4];
#pragma unroll
            for (int v4 = 0; v4 < 4; ++v4) ya[v4] = yp[v4];
            // the next row's pair bit (bit r-1 of pbn; 0 after the last row) and lane 31's left value
            const int bn = (int)(((pbn << 1) >> r) & 1u);
            const int ln = (int)ws.left[r] + bn;
            // the terms that do not go through the closure: the split k = i+1 (D(i,i) + D(i+1,j))
            // and the old terms
            int y = max(yold, below);
            y = valid ? y : kNeg16;
            // old terms of the next row overlap with this closure (the last one is unused)
            yold = old_terms(max(r - 1, 0));
            unsigned a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint4 a = ya[v];
                a0 = __viaddmax_s16x2(a.x, Wp[4 * v + 0], a0);
                a1 = __viaddmax_s16x2(a.y, Wp[4 * v + 1], a1);
                a2 = __viaddmax_s16x2(a.z, Wp[4 * v + 2], a2);
                a3 = __viaddmax_s16x2(a.w, Wp[4 * v + 3], a3);
            }
            const unsigned acc = __vmaxs2(__vmaxs2(a0, a1), __vmaxs2(a2, a3));
            int d = max(y, hmax2(acc));
            d = valid ? d : 0;
            // the next row's exchanged value, ordered before the row's other stores (after the last
            // row it lands in the buffer the next tile fills first)
            ws.y[(r - 1) & 1][yslot] = (int16_t)(c == 31 ? ln : d + bn);
            __syncwarp();
            publish(r, d, below);
            below = d;
            if constexpr (TV) {
                // the window moves down one row: value e+1 <- value e, value 0 <- d
#pragma unroll
                for (int e = WS::NWP - 1; e > 0; --e) wpk[e] = __byte_perm(wpk[e - 1], wpk[e], 0x5432);
                wpk[0] = __byte_perm((unsigned)d, wpk[0], 0x5410);
            }
        }
    }
    __syncwarp();
    if (P.trace) tdeps[2] = (long long)gtimer();
    // column mode: the next tile's chunk counter, read now and acquired by the fence that releases
    // this tile
    int cnt_next = 0;
    if constexpr (COL) {
        if (lane == 0 && nn_next > 0) cnt_next = ld_relaxed(P.cnt + sd.cnt_off + (I - 1) * NT + J);
    }
    // the row features of (I,J) are read by the middle blocks K = J of later tiles (I, J' > J) only:
    // none in the last tile column, which is the fold's critical chain
    if constexpr (TV) {
      if (J + 1 < NT) {
        bool up[T];
        int av[T];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            const int d = (int)tile[r][c];
            const int dl = (int)tile[r][c > 0 ? c - 1 : 0];
            up[r] = (d - dl) == 1;
            av[r] = (int)tile[r][(c < G) ? c * Q : 0];
        }
        unsigned hb[T];
#pragma unroll
        for (int r = 0; r < T; ++r) hb[r] = __ballot_sync(FULL, up[r]);
        if (c < G) {
#pragma unroll
            for (int r = 0; r < T; ++r) {
                const uint32_t f = ((uint32_t)av[r] << 16) | ((hb[r] >> (c * Q + 1)) & C::BMASK);
                P.rf[sd.rf_off + (size_t)(IT + r) * NG + J * G + c] = f;
                if constexpr (COL) {
                    if (cs.consumer) ws.rfo[buf][r][c] = f;
                }
            }
        }
      }
    }
    if constexpr (COL) {
        // the tile (and its row features) is complete in shared memory: hand it to the next column's
        // warp before the slower global copies and the release below
        if (cs.consumer) {
            __syncwarp();
            if (lane == 0) st_release_cta(&ws.produced, cs.k + 1);
        }
    }
    // ---- column-major copy (lane = row); two-vector column mode reads columns only as features, and
    // the other two-vector tiles read one column of it: the left neighbour's last, D(i, JT-1)
    if (lane < T && !(COL && TV)) {
        if constexpr (TV) {
            Dcol[(size_t)(JT + T - 1) * PC + IT + lane + kColOff] = tile[lane][T - 1];
        } else {
#pragma unroll 8
            for (int cc = 0; cc < T; ++cc) Dcol[(size_t)(JT + cc) * PC + IT + lane + kColOff] = tile[lane][cc];
        }
    }
    // answer D(0, n-1); on the serving ring it goes to host memory, after a system-scope fence that
    // makes the table (this warp's rows, and the other tiles it acquired) visible to the host's copies
    if (I == 0 && J == NT - 1) {
        const int cn = (sd.n - 1) - JT;
        if (P.ring_cap > 0) __syncwarp();
        if (sd.n >= 1 && lane == cn) {
            const int v = (sd.n >= 2) ? (int)tile[0][cn] : 0;
            if (P.ring_cap > 0) {
                __threadfence_system();
                *(volatile int *)(P.results + sd.result_index) = v;
            } else {
                P.results[sd.result_index] = v;
            }
        }
    }
    if constexpr (COL) {
        // carry the column's constants and the bottom row to the next tile of this column
        if (cs.k == 0) {
#pragma unroll
            for (int mm = 0; mm < 16; ++mm) {
                const int c0 = 2 * mm, c1 = 2 * mm + 1;
                const int w0 = (valid && c0 < c) ? (int)tile[min(c0 + 1, T)][c] : (valid && c0 == c) ? 0 : kNeg16;
                const int w1 = (valid && c1 < c) ? (int)tile[min(c1 + 1, T)][c] : (valid && c1 == c) ? 0 : kNeg16;
                cs.Wp[mm] = (unsigned)(w0 & 0xffff) | ((unsigned)w1 << 16);
            }
        }
        if (cs.k == 1) {
            if constexpr (TV) {
#pragma unroll
                for (int gl = 0; gl < G; ++gl) {
                    const uint32_t cf = ws.cbc[c][gl];
                    cs.lcb0[gl] = cf;
                }
            } else {
#pragma unroll
                for (int w = 0; w < 16; ++w)
                    cs.lcol0[w] = (unsigned)(uint16_t)tile[1 + 2 * w][c] | ((unsigned)(uint16_t)tile[2 + 2 * w][c] << 16);
            }
        }
        cs.colT = below;
    }
    if (P.trace) tdeps[3] = (long long)gtimer();
    // every lane's stores are ordered before lane 0's release by the warp barrier; the release is
    // cumulative, so a reader that acquires the flag sees the whole tile
    __syncwarp();
    if constexpr (COL) {
        // one fence serves as this tile's release and as the acquire of the next tile's chunk
        // counter, read just before it
        int seen = 0;
        if (lane == 0) {
            fence_acq_rel();
            st_relaxed(flags + I * NT + J, 1);
            seen = (nn_next > 0 && cnt_next >= nn_next) ? 1 : 0;
        }
        cs.cnt_ok = __shfl_sync(FULL, seen, 0) != 0;
        cs.failed = false;
        __syncwarp();
    } else {
        if (lane == 0) st_release(flags + I * NT + J, 1);
    }
    return tfar;
}

}  // namespace fold

#include "fold_column.cuh"

namespace fold {

// ---------------------------------------------------------------- kernel
// MEMO: Section 3.2's partially memoised variant (R rows tabulated on first sight in each CTA)
template <int Q, int M, bool MEMO>
__global__ void __launch_bounds__(kThreads, 1) fold_kernel(FoldParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    using C = Cfg<Q, M>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *Rs = smem;
    if constexpr (MEMO && memo_words<Q, M>() > 0) {
        // memoised R: no table yet, no row tabulated
        unsigned *bits = reinterpret_cast<unsigned *>(smem + memo_offset<Q, M>());
        for (int v = threadIdx.x; v < memo_words<Q, M>(); v += blockDim.x) bits[v] = 0u;
    } else if constexpr (C::RBYTES > 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.rtab);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        // the device copy of R is padded to a multiple of 256 bytes, so rounding up stays in bounds
        for (int v = threadIdx.x; v < (C::RBYTES + 15) / 16; v += blockDim.x) dst[v] = __ldg(src + v);
    }
    WarpScratch<Q, M> *wsb = reinterpret_cast<WarpScratch<Q, M> *>(smem + round_up(C::RBYTES, 128));
    WarpScratch<Q, M> &ws = wsb[warp];
    if (lane == 0) {
        ws.produced = 0;
        ws.consumed = 0;
    }
    constexpr int kHalf = kWarpsPerCta / 2;
    constexpr bool kHelp = (M == kTwoVector) && col_helpers_fit<Q>();
    if constexpr (kHelp) {
        if (P.col_helpers && warp >= kHalf && lane == 0) {
            ColHelp<Q> *ha = reinterpret_cast<ColHelp<Q> *>(&ws);
            ha->mprog = 0;
            ha->prep_ready = 0;
            ha->consumed = 0;
        }
    }
    __syncthreads();
    const bool split = P.near_ctas > 0;
    const bool far_role = split && (int)blockIdx.x >= P.near_ctas;
    // column mode: once every column of a tile CTA is finished, its warps take chunk tasks with the
    // chunk CTAs (P.col_join): the left columns finish first, while the middle diagonals' chunk work is
    // at its largest.  The CTA is finished when the last tile of its rightmost column, (0, Jr), is
    // published: that tile waited for (0, Jr-1), read from the neighbour's shared buffers, and so on
    // down the CTA's columns, so no warp of the CTA reads another's shared memory any more.
    // The wait may last nearly the whole fold (the first tile CTA holds the last column), so it is
    // not an error when it outlasts the wait bound: the warp then just leaves without joining.
    bool joined = false;
    auto join_chunks = [&](int Jr) -> bool {
        if (Jr < 0) return true;
        const int *flag = P.flags + P.seqs[0].flag_off + Jr;
        int ok = 0;
        if (lane == 0) {
            const unsigned long long t0 = gtimer();
            unsigned ns = 64;
            for (;;) {
                if (ld_acquire(flag) >= 1) { ok = 1; break; }
                if (*(volatile int *)P.error != 0 || (long long)(gtimer() - t0) > P.timeout_ns) break;
                __nanosleep(ns);
                ns = ns < 1024 ? 2 * ns : 1024;
            }
        }
        ok = __shfl_sync(FULL, ok, 0);
        __syncwarp();
        return ok != 0;
    };
    if constexpr (kHelp) {
        if (P.col_mode && P.col_helpers && split && !far_role) {
            // column mode with helpers: warp w < kHalf computes the rows of tile column J, warp
            // w + kHalf is its helper (fold_column.cuh)
            const SeqDesc sd = P.seqs[0];
            const int NT = sd.NT;
            const int cpc = P.cols_per_cta;
            const int col_ctas = (NT + cpc - 1) / cpc;
            const bool main_role = warp < kHalf;
            const int w = main_role ? warp : warp - kHalf;
            const int base = (col_ctas - 1 - (int)blockIdx.x) * cpc;
            const int J = base + w;
            const int ncols = ((int)blockIdx.x < col_ctas && cpc <= kHalf) ? max(0, min(cpc, NT - base)) : 0;
            bool ok = true;
            if (w < ncols) {
                ColHelp<Q> &ha = *reinterpret_cast<ColHelp<Q> *>(&wsb[w + kHalf]);
                const bool consumer = (w + 1 < cpc) && (J + 1 < NT);
                if (main_role) {
                    ColMain<Q> cs;
#pragma unroll
                    for (int mm = 0; mm < 16; ++mm) cs.Wp[mm] = 0u;
                    cs.colT = 0;
                    cs.consumer = consumer;
                    for (int k = 0; k <= J; ++k) {
                        const int I = J - k;
                        const int idx = k * NT - k * (k - 1) / 2 + I;
                        long long t0 = 0, tt[2] = {0, 0};
                        if (P.trace && lane == 0) t0 = (long long)gtimer();
                        const int nfar = k >= 1 ? P.tasks[idx].z : 0;
                        const bool tok = col_main_tile<Q, MEMO>(P, sd, I, J, k, nfar, wsb[w], ha, Rs, lane, cs,
                                                                P.trace ? tt : nullptr);
                        if (P.trace && lane == 0 && tok) {
                            long long *rec = P.trace + (size_t)idx * kTraceWords;
                            rec[0] = ((long long)(blockIdx.x * kWarpsPerCta + warp) << 32) | (unsigned)idx;
                            rec[1] = ((long long)kTaskNear << 32) | 0u;
                            rec[2] = ((long long)I << 32) | (unsigned)J;
                            rec[3] = t0;
                            rec[4] = tt[0];
                            rec[5] = tt[0];
                            rec[6] = (long long)gtimer();
                            rec[7] = tt[0];
                            rec[8] = tt[1];
                            rec[9] = tt[1];
                            rec[10] = (long long)smid();
                        }
                        if (!tok) {
                            ok = false;
                            break;
                        }
                    }
                } else {
                    ColHelper<Q> hs;
                    hs.have_lcb0 = false;
                    hs.sj = lane < Cfg<Q, M>::T ? (int)P.codes[sd.code_off + J * Cfg<Q, M>::T + lane] : kPadCode;
                    WarpScratch<Q, M> *prodM = w > 0 ? &wsb[w - 1] : nullptr;
                    ColHelp<Q> *prodH = w > 0 ? reinterpret_cast<ColHelp<Q> *>(&wsb[w - 1 + kHalf]) : nullptr;
                    for (int k = 0; k <= J; ++k)
                        if (!col_help_prep<Q, MEMO>(P, sd, J - k, J, k, wsb[w], ha, prodM, prodH, Rs, lane, hs)) {
                            ok = false;
                            break;
                        }
                }
            }
            if (!P.col_join || !ok || (int)blockIdx.x >= col_ctas) return;
            if (!join_chunks(base + ncols - 1)) return;
            joined = true;
        }
    }
    if (P.col_mode && split && !far_role && !joined) {
        // column mode: this warp computes the tiles of one column, bottom-up
        const SeqDesc sd = P.seqs[0];
        const int NT = sd.NT;
        // the longest columns (the right end, whose chains set the fold's time) go to the CTAs
        // launched first, away from the chunk CTAs that follow the tile CTAs in launch order
        const int col_ctas = (NT + P.cols_per_cta - 1) / P.cols_per_cta;
        const int base = (col_ctas - 1 - (int)blockIdx.x) * P.cols_per_cta;
        const int J = base + warp;
        const int ncols = (int)blockIdx.x < col_ctas ? max(0, min(P.cols_per_cta, NT - base)) : 0;
        bool failed = false;
        if (warp < ncols) {
            NearCol<Q, M> cs;
            cs.prod = warp > 0 ? &wsb[warp - 1] : nullptr;
            cs.consumer = (warp + 1 < P.cols_per_cta) && (J + 1 < NT);
            cs.colT = 0;
            cs.cnt_ok = false;
            cs.tasks = P.tasks;
            for (int k = 0; k <= J; ++k) {
                const int I = J - k;
                cs.k = k;
                const int idx = k * NT - k * (k - 1) / 2 + I;   // tile (I,J) in the diagonal-ordered tile tasks
                const int4 tk = P.tasks[idx];
                long long t0 = 0, tdeps[4] = {0, 0, 0, 0};
                if (P.trace && lane == 0) t0 = (long long)gtimer();
                const long long tmid = run_near<Q, M, true, MEMO>(P, sd, I, J, tk.z, ws, Rs, lane, tdeps, cs);
                if (P.trace && lane == 0) {
                    long long *rec = P.trace + (size_t)idx * kTraceWords;
                    rec[0] = ((long long)(blockIdx.x * kWarpsPerCta + warp) << 32) | (unsigned)idx;
                    rec[1] = ((long long)kTaskNear << 32) | (unsigned)tk.x;
                    rec[2] = ((long long)I << 32) | (unsigned)J;
                    rec[3] = t0;
                    rec[4] = tdeps[0];
                    rec[5] = tmid;
                    rec[6] = (long long)gtimer();
                    rec[7] = tdeps[1];
                    rec[8] = tdeps[2];
                    rec[9] = tdeps[3];
                    rec[10] = (long long)smid();
                }
                if (cs.failed) break;   // a wait gave up (its error is in P.error)
            }
            failed = cs.failed;
        }
        if (!P.col_join || failed || (int)blockIdx.x >= col_ctas) return;
        if (!join_chunks(base + ncols - 1)) return;
        joined = true;
    }
    const bool chunk_role = far_role || joined;
    NextTask nt;
    nt.qhead = chunk_role ? P.queue_head_far : P.queue_head;
    nt.qbase = chunk_role ? P.nnear : 0;
    nt.qlimit = P.ring_cap > 0 ? 0x7fffffff : ((split && !chunk_role) ? P.nnear : P.ntasks);
    nt.tasks = P.tasks;
    nt.have = false;
    nt.stopped = false;
    nt.ring_cap = P.ring_cap;
    nt.ring_tail = P.ring_tail;
    nt.ring_stop = P.ring_stop;
    nt.ring_progress = P.ring_progress;
    nt.error = P.error;
    nt.timeout_ns = P.timeout_ns;
    int err = 0;   // the error word as read when the previous task started
    for (;;) {
        if (!nt.have) nt.claim(lane);
        nt.have = false;
        nt.fetch(lane);
        const int idx = nt.idx;
        const int4 tk = nt.tk;
        if (idx >= nt.qlimit || err != 0 || nt.stopped) break;
        err = ld_relaxed(P.error);   // checked before the next task
        const SeqDesc sd = P.seqs[tk.x];
        const int I = task_I(tk.y), J = task_J(tk.y);
        long long t0 = 0, tdeps[4] = {0, 0, 0, 0};
        if (P.trace && lane == 0) t0 = (long long)gtimer();
        long long tmid;
        const int ty = task_type(tk.y);
        if (ty == kTaskNear) {
            NearCol<Q, M> none;
            none.k = 0;
            none.prod = nullptr;
            none.consumer = false;
            none.cnt_ok = false;
            tmid = run_near<Q, M, false, MEMO>(P, sd, I, J, tk.z, ws, Rs, lane, tdeps, none);
        }
        else if (ty == kTaskFar) tmid = run_far<Q, M, MEMO>(P, sd, I, J, tk.z, tk.w, ws, Rs, lane, tdeps, nt);
        else tmid = run_far_strip<Q, M, MEMO>(P, sd, I, J, tk.z, tk.w, ws, Rs, lane, tdeps, nt);
        if (P.trace && lane == 0) {
            long long *rec = P.trace + (size_t)idx * kTraceWords;
            rec[0] = ((long long)(blockIdx.x * kWarpsPerCta + warp) << 32) | (unsigned)idx;
            rec[1] = ((long long)task_type(tk.y) << 32) | (unsigned)tk.x;
            rec[2] = ((long long)I << 32) | (unsigned)J;
            rec[3] = t0;
            rec[4] = tdeps[0];
            rec[5] = tmid;
            rec[6] = (long long)gtimer();
            rec[7] = tdeps[1];
            rec[8] = tdeps[2];
            rec[9] = tdeps[3];
            rec[10] = (long long)smid();
        }
    }
}

template <int Q, int M, bool MEMO = false>
inline cudaError_t launch_q(const FoldParams &p, int grid, cudaStream_t st) {
    size_t sm = smem_bytes_for<Q, M>();
    cudaError_t e = cudaFuncSetAttribute(fold_kernel<Q, M, MEMO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    fold_kernel<Q, M, MEMO><<<grid, kThreads, sm, st>>>(p);
    return cudaGetLastError();
}

template <int Q, int M>
inline int blocks_per_sm_q() {
    int nb = 0;
    size_t sm = smem_bytes_for<Q, M>();
    if (cudaFuncSetAttribute(fold_kernel<Q, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fold_kernel<Q, M, false>, kThreads, sm) != cudaSuccess) return 0;
    return nb;
}

}  // namespace fold
