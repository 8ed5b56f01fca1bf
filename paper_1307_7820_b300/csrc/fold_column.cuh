// fold_column.cuh -- column mode with a helper warp per tile column (two-vector, single folds).
// Included by fold_kernel.cuh after the NEAR task; uses its helpers.
//
// In column mode warp w of a tile CTA owns tile column J and computes its tiles bottom-up, (J,J)
// first; the fold's time is the chain of those tiles in the last column (one tile per tile
// diagonal).  Here that warp (the main warp) keeps the rows -- pair term, residual splits, the tile
// column's own groups and the closure (Section 3.1, Eq. 1 and Eq. 3) -- and the tile's publication,
// and a helper warp w + kWarpsPerCta/2 of the same CTA prepares each next tile (I,J):
//
//   A. loads its old inputs once their flags are set: the row words of the diagonal tile (I,I)
//      and of (I,I+1), the residual splits' D(i,k-1) and the pair bits, into a double-buffered
//      prep area;
//   B. does the lookups of middle block K = J-1 (the left neighbour (I,J-1)'s row features against
//      the column features of tile (J-1,J), which this column computed second) and copies the left
//      neighbour's last column (the closure's left values);
//   C. merges the chunks' partial maximum of middle blocks I+2 .. J-2 (the P slot) once the tile's
//      chunk counter is complete;
//   D. does the lookups of middle block K = I+1 (the row features of (I,I+1) against the column
//      features of tile (I+1,J), this column's previous tile);
//   and publishes the prep -- the far partial maximum of every cell -- to the main warp.
//
// B and D run step by step while their producers compute: the left neighbour is the previous
// column's tile k-1 and the bottom neighbour this column's tile k-1, computed at about the same
// time by the two main warps, which publish a progress count after every group of q rows; after
// each step the helper takes the rows (B: their features from one ballot per row of the producer's
// tile buffer) and the group of column features (D) completed so far.  C is polled between the
// steps.  So the main warp waits only for the last row's work after its previous tile, and the
// old-input loads, the late blocks' lookups and the chunk merge overlap the rows.  When the left
// neighbour runs in another CTA, B waits for its flag and reads it from global memory.
//
// Ordering.  Main and helper synchronise through shared words with CTA-scope release/acquire:
// mprog (main: (G+1) steps per tile -- one per completed group of column features, one when the
// tile is done), prep_ready (helper: tiles whose prep is complete) and consumed (written by the next
// column's helper: tiles of this column it has read; the main warp reuses a tile buffer two tiles
// later only after that).  Each main warp releases its own tile to other CTAs (row features, the
// P slot cleared for its next user, one gpu-scope fence and the flag), so every global store is
// fenced by the warp that made it.  Every wait is bounded.
#pragma once

namespace fold {

// The prep of one tile (I,J), written by the helper, read by the main warp.
template <int Q>
struct __align__(16) ColPrep {
    using WS = WarpScratch<Q, kTwoVector>;
    static constexpr int T = WS::T;
    alignas(16) uint32_t gw[T][WS::GA];     // per row of (I,I) and group, (A << 16) | R-row offset,
                                            // A = -32768 for groups not complete below that row
    alignas(16) uint32_t rpk[T][WS::NWPA];  // per row, the residual splits' D(i, k-1) as int16 pairs
    alignas(16) int16_t pm[T][32];          // far partial maximum of each cell (P and blocks J-1, I+1)
    unsigned pbits[32];                     // per lane (column), pair bits against the tile's rows
    int16_t left[T + 2];                    // left[m] = D(IT+m, JT-1), m = 1..T; left[0] = 0
};

// The helper's shared area (it overlays the helper warp's WarpScratch).
template <int Q>
struct __align__(16) ColHelp {
    using WS = WarpScratch<Q, kTwoVector>;
    static constexpr int T = WS::T;
    ColPrep<Q> prep[2];
    alignas(16) uint32_t lrf[2][T][WS::GA];  // staged row words: [0] tile (I,J-1) (block J-1),
                                             // [1] tile (I,I+1) (block I+1)
    alignas(16) uint32_t lcb0[32][WS::GA];   // column features of tile (J-1,J), set by the main warp
    int mprog;
    int prep_ready;
    int consumed;
};

template <int Q>
__host__ __device__ constexpr bool col_helpers_fit() {
    return sizeof(ColHelp<Q>) <= sizeof(WarpScratch<Q, kTwoVector>);
}

// ---------------------------------------------------------------- main warp
template <int Q>
struct ColMain {
    unsigned Wp[16];   // packed W[c'][c] of tile (J,J) (set by tile 0)
    int colT;          // D(IT, j) of the tile just finished (row 0), the next tile's bottom neighbour
    int sj;            // code of this lane's column base
    bool consumer;     // the next column's warps run in this CTA
};

// Main warp, before a tile: waits (bounded) until the helper has published the tile's prep
// (*prep >= target) and, with nfar > 0, until the tile's chunk counter reaches nfar, starting the
// copy of the P slot (nints ints) into dst as soon as it does; the counter is polled every fourth
// round, so the prep is seen within a few shared-memory round trips.  Returns false if a wait gave
// up (no copy is then left in flight).
static __device__ __noinline__ bool wait_prep_and_slot(const int *prep, int target, const int *cnt, int nfar,
                                                       const int *slot, int *dst, int nints, int *error,
                                                       long long timeout_ns, int lane) {
    bool have_p = nfar <= 0, have_prep = false;
    const unsigned long long t0 = gtimer();
    for (unsigned it = 0;; ++it) {
        if (!have_p && (it & 3u) == 0) {
            int v = 0;
            if (lane == 0) v = ld_acquire(cnt);
            if (__shfl_sync(FULL, v, 0) >= nfar) {
                __syncwarp();   // every lane's copy after lane 0's acquire
                for (int q = lane; q < nints / 4; q += 32)
                    cp_async16(reinterpret_cast<int4 *>(dst) + q, reinterpret_cast<const int4 *>(slot) + q);
                cp_async_commit();
                have_p = true;
            }
        }
        if (!have_prep) {
            int v = 0;
            if (lane == 0) v = ld_acquire_cta(prep);
            have_prep = __shfl_sync(FULL, v, 0) >= target;
        }
        if (have_p && have_prep) break;
        if ((it & 31u) == 31u) {
            int bad = 0;
            if (lane == 0) {
                if (*(volatile int *)error != 0) bad = 1;
                else if ((long long)(gtimer() - t0) > timeout_ns) {
                    atomicCAS(error, 0, kErrTimeout);
                    bad = 1;
                }
            }
            if (__shfl_sync(FULL, bad, 0)) {
                cp_async_wait_all();
                __syncwarp();
                return false;
            }
        }
    }
    cp_async_wait_all();
    __syncwarp();
    return true;
}

// Tile (I,J) = the column's k-th tile, t = J - I = k.  Returns false if a wait gave up.
template <int Q, bool MEMO>
__device__ __forceinline__ bool col_main_tile(const FoldParams &P, const SeqDesc &sd, int I, int J, int k, int nfar,
                                              WarpScratch<Q, kTwoVector> &ws, ColHelp<Q> &ha, const uint8_t *Rs,
                                              int lane, ColMain<Q> &cs, long long *tr) {
    using C = Cfg<Q, kTwoVector>;
    using WS = WarpScratch<Q, kTwoVector>;
    constexpr int T = C::T, G = C::G;
    const int NT = sd.NT, Np = sd.Np;
    const int t = k;
    const int IT = I * T, JT = J * T;
    const int c = lane;
    const bool valid = c < T;
    const int j = JT + c;
    int16_t *Drow = P.drow + sd.drow_off;
    int16_t(*tile)[33] = (k & 1) ? ws.tile1 : ws.tile;
    // the next column's helper must have read this column's tile k-2 before its buffer is rewritten
    if (cs.consumer && k >= 2 && !wait_smem_geq(&ha.consumed, k - 1, P.error, P.timeout_ns, lane)) return false;
    // the helper's prep, and the chunks' partial maximum of the middle blocks I+2 .. J-2 (the P
    // slot), copied into shared memory as soon as the tile's chunk counter is complete
    const int *pslot = P.pring + sd.p_off + ((size_t)(t % kRing) * NT + I) * (T * T);
    constexpr bool PB = WS::PB;   // else the helper merges the slot into the prep
    if (!wait_prep_and_slot(&ha.prep_ready, k + 1, P.cnt + sd.cnt_off + I * NT + J, PB ? nfar : 0, pslot, ws.pbuf,
                            PB ? T * T : 0, P.error, P.timeout_ns, lane))
        return false;
    if (tr) tr[0] = (long long)gtimer();
    const ColPrep<Q> &pp = ha.prep[k & 1];
    const unsigned pbits = pp.pbits[lane];
    const int colT = cs.colT;
    if (valid) tile[T][c] = (int16_t)colT;
    // this tile's column groups start as (B, c) = (0, 0): a group that is not complete below a row
    // then adds at most -32768 + q - 1 there (its A is -32768)
#pragma unroll
    for (int g4 = 0; g4 < WS::GA / 4; ++g4)
        reinterpret_cast<uint4 *>(&ws.cbc[c][0])[g4] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();

    const int ms_base = (G + 1) * k;   // progress count before this tile
    int ms_row = (G - 1) * Q + 1;      // next row that completes a group of column features (rows go
                                       // bottom-up, so group G-1 completes first and group 0 last)
    unsigned vhist = 0;                // vertical differences, newest in bit 0
    unsigned wpk[WS::NWP];             // residual window: value e = D(IT+r+1+e, j), int16 pairs
#pragma unroll
    for (int e = 0; e < WS::NWP; ++e) wpk[e] = 0u;
    wpk[0] = (unsigned)colT & 0xffffu;

    // publishes row r: tile copy, row-major store, column features; and the progress count after a
    // completed group of column features (the helper's lookups of block I+1 for the next tile)
    uint32_t *rf_tile = P.rf + sd.rf_off + (size_t)IT * (Np / Q) + J * G;
    auto publish = [&](int r, int d, int below_prev) {
        tile[r][c] = (int16_t)d;
        if (T == 32 || valid) Drow[(size_t)(IT + r) * Np + j] = (int16_t)d;
        const int vb = d - below_prev;   // vertical difference D(i,j) - D(i+1,j)
        vhist = (vhist << 1) | (unsigned)(vb & 1);
        if (r == ms_row) {
            const int gl = (r - 1) / Q;
            const uint32_t cb = ((uint32_t)d << 16) | (vhist & C::BMASK);
            ws.cbc[c][gl] = cb;
            if (valid) P.cf[sd.cf_off + (size_t)(I * G + gl) * Np + j] = cb;
            __syncwarp();
            if (lane == 0) st_release_cta(&ha.mprog, ms_base + (G - gl));
            ms_row -= Q;
        }
    };

    int below = colT;   // D(i+1, j)
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
        // terms of row rr that do not depend on row rr+1 (see run_near): the prep's far partial
        // maximum, the residual splits in the window of rows below, the full groups of tile column I
        auto old_terms = [&](int rr) -> int {
            int best = (int)pp.pm[rr][c];
            if (PB && nfar > 0) best = max(best, ws.pbuf[min(rr * T + c, T * T - 1)]);
            unsigned ra = 0u, rb = 0u;
#pragma unroll
            for (int k4 = 0; k4 < WS::NWPA / 4; ++k4) {
                const uint4 a = reinterpret_cast<const uint4 *>(&pp.rpk[rr][0])[k4];
                if (4 * k4 + 0 < WS::NWP) ra = __viaddmax_s16x2(a.x, wpk[min(4 * k4 + 0, WS::NWP - 1)], ra);
                if (4 * k4 + 1 < WS::NWP) rb = __viaddmax_s16x2(a.y, wpk[min(4 * k4 + 1, WS::NWP - 1)], rb);
                if (4 * k4 + 2 < WS::NWP) ra = __viaddmax_s16x2(a.z, wpk[min(4 * k4 + 2, WS::NWP - 1)], ra);
                if (4 * k4 + 3 < WS::NWP) rb = __viaddmax_s16x2(a.w, wpk[min(4 * k4 + 3, WS::NWP - 1)], rb);
            }
            best = max(best, hmax2(__vmaxs2(ra, rb)));
            int gm = (int)0x80000000u;
#pragma unroll
            for (int g4 = 0; g4 < WS::GA / 4; ++g4) {
                const uint4 gv = reinterpret_cast<const uint4 *>(&pp.gw[rr][0])[g4];
                const uint4 cv = reinterpret_cast<const uint4 *>(&ws.cbc[c][0])[g4];
                if (4 * g4 + 0 < G) gm = max(gm, group_term<Q>(Rs, gv.x, cv.x));
                if (4 * g4 + 1 < G) gm = max(gm, group_term<Q>(Rs, gv.y, cv.y));
                if (4 * g4 + 2 < G) gm = max(gm, group_term<Q>(Rs, gv.z, cv.z));
                if (4 * g4 + 3 < G) gm = max(gm, group_term<Q>(Rs, gv.w, cv.w));
            }
            return max(best, gm >> 16);
        };
        int yold = old_terms(T - 1);
        // the closure exchange (see run_near): lane c'-1 stores its value of the row below plus
        // column c''s pair bit at position c', lane 31 the left column's value at position 0
        const unsigned pbn = __shfl_sync(FULL, pbits, (lane + 1) & 31);   // column c+1's pair bits
        const int yslot = (c + 1) & 31;
        {
            const int bv = c == 31 ? (int)pp.left[T] : colT;
            ws.y[(T - 1) & 1][yslot] = (int16_t)(bv + (int)((pbn >> (T - 1)) & 1u));
        }
        __syncwarp();
        const unsigned *Wp = cs.Wp;
#pragma unroll 2
        for (int r = T - 1; r >= 0; --r) {
            const uint4 *yp = reinterpret_cast<const uint4 *>(ws.y[r & 1]);
            uint4 ya[4];
#pragma unroll
            for (int v4 = 0; v4 < 4; ++v4) ya[v4] = yp[v4];
            const int bn = (int)(((pbn << 1) >> r) & 1u);
            const int ln = (int)pp.left[r] + bn;
            int y = max(yold, below);
            y = valid ? y : kNeg16;
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
            ws.y[(r - 1) & 1][yslot] = (int16_t)(c == 31 ? ln : d + bn);
            __syncwarp();
            publish(r, d, below);
            below = d;
#pragma unroll
            for (int e = WS::NWP - 1; e > 0; --e) wpk[e] = __byte_perm(wpk[e - 1], wpk[e], 0x5432);
            wpk[0] = __byte_perm((unsigned)d, wpk[0], 0x5410);
        }
    }
    __syncwarp();
    if (tr) tr[1] = (long long)gtimer();
    if (k == 0) {
#pragma unroll
        for (int mm = 0; mm < 16; ++mm) {
            const int c0 = 2 * mm, c1 = 2 * mm + 1;
            const int w0 = (valid && c0 < c) ? (int)tile[min(c0 + 1, T)][c] : (valid && c0 == c) ? 0 : kNeg16;
            const int w1 = (valid && c1 < c) ? (int)tile[min(c1 + 1, T)][c] : (valid && c1 == c) ? 0 : kNeg16;
            cs.Wp[mm] = (unsigned)(w0 & 0xffff) | ((unsigned)w1 << 16);
        }
    }
    if (k == 1) {   // the column features of tile (J-1,J), for the helper's block J-1 lookups
#pragma unroll
        for (int g4 = 0; g4 < WS::GA / 4; ++g4)
            reinterpret_cast<uint4 *>(&ha.lcb0[c][0])[g4] = reinterpret_cast<const uint4 *>(&ws.cbc[c][0])[g4];
    }
    // answer D(0, n-1)
    if (I == 0 && J == NT - 1) {
        const int cn = (sd.n - 1) - JT;
        if (sd.n >= 1 && lane == cn) P.results[sd.result_index] = (sd.n >= 2) ? (int)tile[0][cn] : 0;
    }
    cs.colT = below;
    // the tile is complete in shared memory: the helpers (this column's, for the next tile's block
    // I+1 lookups, and the next column's, for its left neighbour) may read it
    __syncwarp();
    if (lane == 0) st_release_cta(&ha.mprog, ms_base + G + 1);
    // the tile's row features (one ballot per row; horizontal vectors, Section 3.1), its P slot
    // cleared for tile (I, J+kRing) (the helper read it before publishing this tile's prep), and its
    // release: this warp's fence covers its own global stores of the tile.  The row features are
    // read only by later tiles of row I, so not in the last column (the critical chain); the slot
    // only if a tile (I, J+kRing) exists
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
            for (int r = 0; r < T; ++r)
                rf_tile[(size_t)r * (Np / Q) + c] = ((uint32_t)av[r] << 16) | ((hb[r] >> (c * Q + 1)) & C::BMASK);
        }
    }
    {
        if (nfar > 0 && J + kRing < NT) {
            int *slot = P.pring + sd.p_off + ((size_t)(t % kRing) * NT + I) * (T * T);
            if constexpr ((T * T) % 4 == 0) {
#pragma unroll
                for (int q4 = lane; q4 < T * T / 4; q4 += 32) __stcg(reinterpret_cast<int4 *>(slot) + q4, make_int4(0, 0, 0, 0));
            } else if (valid) {
#pragma unroll
                for (int r = 0; r < T; ++r) __stcg(slot + r * T + c, 0);
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        fence_acq_rel();
        st_relaxed(P.flags + sd.flag_off + I * NT + J, 1);
    }
    __syncwarp();
    return true;
}

// ---------------------------------------------------------------- helper warp
template <int Q>
struct ColHelper {
    static constexpr int G = Cfg<Q, kTwoVector>::G;
    uint32_t lcb0[G];   // column features of tile (J-1,J) in this lane's column (from tile k = 2 on)
    bool have_lcb0;
    int sj;             // code of this lane's column base
};

// A-D: the prep of tile (I,J) = the column's k-th tile.
template <int Q, bool MEMO>
__device__ __forceinline__ bool col_help_prep(const FoldParams &P, const SeqDesc &sd, int I, int J, int k,
                                              WarpScratch<Q, kTwoVector> &wm, ColHelp<Q> &ha,
                                              WarpScratch<Q, kTwoVector> *prodM, ColHelp<Q> *prodH,
                                              const uint8_t *Rs, int lane, ColHelper<Q> &hs) {
    using C = Cfg<Q, kTwoVector>;
    using WS = WarpScratch<Q, kTwoVector>;
    constexpr int T = C::T, G = C::G;
    constexpr int E = (T * G + 31) / 32;
    const int NT = sd.NT, Np = sd.Np, NG = Np / Q;
    const int t = k;
    const int IT = I * T, JT = J * T;
    const int c = lane;
    const bool valid = c < T;
    const int16_t *Drow = P.drow + sd.drow_off;
    const uint8_t *codes = P.codes + sd.code_off;
    const uint32_t *RF = P.rf + sd.rf_off;
    const bool lateA = t >= 2, lateB = t >= 3;
    ColPrep<Q> &pp = ha.prep[k & 1];

    // ---- A: old inputs
    {
        const int rcode = lane < T ? (int)codes[IT + lane] : kPadCode;
        unsigned pbx[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) pbx[x] = __ballot_sync(FULL, (P.pair64 >> (8 * rcode + x)) & 1ull);
        const int sj = hs.sj;
        pp.pbits[lane] = sj == 0 ? pbx[0] : sj == 1 ? pbx[1] : sj == 2 ? pbx[2] : sj == 3 ? pbx[3] : 0u;
    }
    if (t >= 1) {
        // the old tiles read here, (I,I) and (I,I+1), are published by other columns' helpers
        if (!warp_wait_flags(P.flags + sd.flag_off + I * NT + I, lateB ? P.flags + sd.flag_off + I * NT + (I + 1) : nullptr,
                             nullptr, P, lane))
            return false;
        uint32_t fv[E], fb[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = e * 32 + lane;
            const bool in = idx < T * G;
            const size_t row = (size_t)(IT + (in ? idx / G : 0)) * NG;
            fv[e] = in ? __ldcg(RF + row + I * G + idx % G) : 0u;
            fb[e] = (in && lateB) ? __ldcg(RF + row + (I + 1) * G + idx % G) : 0u;
        }
        // residual splits of row rr of the diagonal tile: slot e holds D(IT+rr, IT+kk-1) for
        // kk = rr+2+e while kk is at most the end ce of the first group after the row
        uint32_t w[WS::NWPA];
#pragma unroll
        for (int q4 = 0; q4 < WS::NWPA; ++q4) w[q4] = 0x80008000u;
        if (lane < T) {
            const int rr = lane;
            const int ce = (rr / Q + 1) * Q;
#pragma unroll
            for (int e = 0; e < NW_RES<Q>; ++e) {
                const int kk = rr + 2 + e;
                const uint32_t v = (kk <= ce) ? (uint32_t)(uint16_t)__ldcg(Drow + (size_t)(IT + rr) * Np + IT + min(kk, T) - 1)
                                              : 0x8000u;
                w[e >> 1] = (e & 1) ? ((w[e >> 1] & 0xffffu) | (v << 16)) : ((w[e >> 1] & 0xffff0000u) | v);
            }
#pragma unroll
            for (int k4 = 0; k4 < WS::NWPA / 4; ++k4)
                reinterpret_cast<uint4 *>(&pp.rpk[rr][0])[k4] = make_uint4(w[4 * k4], w[4 * k4 + 1], w[4 * k4 + 2], w[4 * k4 + 3]);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = e * 32 + lane;
            memo_ensure<Q, kTwoVector, MEMO>(Rs, fv[e] & C::BMASK, idx < T * G, lane);
            memo_ensure<Q, kTwoVector, MEMO>(Rs, fb[e] & C::BMASK, idx < T * G && lateB, lane);
            if (idx < T * G) {
                const int rw = idx / G, gl = idx % G;
                const uint32_t hw = C::NIB ? (fv[e] & C::BMASK) : (uint32_t)hrow_offset<Q>((int)(fv[e] & C::BMASK));
                const uint32_t aw = (gl * Q > rw) ? (fv[e] & 0xffff0000u) : 0x80000000u;
                pp.gw[rw][gl] = aw | hw;
                ha.lrf[1][rw][gl] = group_word<Q>(fb[e]);
            }
        }
    }

    // ---- B, C, D: the far partial maximum of every cell of (I,J)
    int acc[T];
#pragma unroll
    for (int r = 0; r < T; ++r) acc[r] = 0;   // scaled by 2^16 (see group_term); every term is >= 0
    if (lateA && !hs.have_lcb0) {
        // the column features of tile (J-1,J), set by this column's main warp at the end of tile 1
        if (!wait_smem_geq(&ha.mprog, (G + 1) * 2, P.error, P.timeout_ns, lane)) return false;
#pragma unroll
        for (int gl = 0; gl < G; ++gl) hs.lcb0[gl] = valid ? ha.lcb0[c][gl] : 0u;
        hs.have_lcb0 = true;
    }
    // C, only where the main warp keeps no shared-memory copy of the P slot (WarpScratch::PB false):
    // the chunks' partial maximum of middle blocks I+2 .. J-2, merged as soon as the tile's chunk
    // counter is seen complete (polled between the steps below, awaited at the end).  Elsewhere the
    // main warp copies the slot itself while it waits for the prep.
    const int idx = t * NT - t * (t - 1) / 2 + I;   // tile (I,J) among the diagonal-ordered tile tasks
    const int nfar = (!WS::PB && t >= 1) ? P.tasks[idx].z : 0;
    bool p_done = nfar == 0;
    const int *cntp = P.cnt + sd.cnt_off + I * NT + J;
    auto merge_p = [&]() {
        const int *slot = P.pring + sd.p_off + ((size_t)(t % kRing) * NT + I) * (T * T);
        int pv[T];
#pragma unroll
        for (int r = 0; r < T; ++r) pv[r] = valid ? __ldcg(slot + r * T + c) : 0;
#pragma unroll
        for (int r = 0; r < T; ++r) acc[r] = max(acc[r], (int)((unsigned)pv[r] << 16));
        p_done = true;
    };
    auto poll_p = [&]() {
        if (p_done) return;
        int v = 0;
        if (lane == 0) v = ld_acquire(cntp);
        if (__shfl_sync(FULL, v, 0) >= nfar) {
            __syncwarp();
            merge_p();
        }
    };
    // B (left neighbour, this CTA) and D (block I+1) step by step: the producer (the previous
    // column's main warp, on tile (I,J-1)) and this column's main warp (on tile (I+1,J)) run at about
    // the same pace; after each completes a group of q rows (its progress count passes a group
    // boundary) the helper does block J-1's lookups for those rows of the producer's tile (their
    // features from one ballot per row) and block I+1's lookups for that group of column features.
    // Step G takes the producer's row 0 and its last column (the closure's left values).
    const int16_t(*pt)[33] = (prodH && t >= 1) ? (((k - 1) & 1) ? prodM->tile1 : prodM->tile) : nullptr;
    const int pbase = (G + 1) * (k - 1);
#pragma unroll
    for (int st = 0; st <= G; ++st) {
        const int m = G - 1 - st;   // group of this step (-1: the producer's tile done)
        if (pt) {
            if (!wait_smem_geq(&prodH->mprog, m >= 0 ? pbase + (G - m) : pbase + G + 1, P.error, P.timeout_ns, lane))
                return false;
            if (lateA) {
                const int r_hi = m == G - 1 ? T - 1 : (m >= 0 ? m * Q + Q : 0);
                const int r_lo = m >= 0 ? m * Q + 1 : 0;
#pragma unroll
                for (int r = T - 1; r >= 0; --r) {
                    if (r > r_hi || r < r_lo) continue;
                    const int d = (int)pt[r][c];
                    const int dl = (int)pt[r][c > 0 ? c - 1 : 0];
                    const unsigned hb = __ballot_sync(FULL, (d - dl) == 1);
                    const int av = (int)pt[r][(c < G) ? c * Q : 0];
                    const uint32_t f = ((uint32_t)av << 16) | ((hb >> ((c < G ? c : 0) * Q + 1)) & C::BMASK);
                    memo_ensure<Q, kTwoVector, MEMO>(Rs, f & C::BMASK, c < G, lane);
                    const uint32_t w = group_word<Q>(f);
#pragma unroll
                    for (int gl = 0; gl < G; ++gl)
                        acc[r] = max(acc[r], group_term<Q>(Rs, __shfl_sync(FULL, w, gl), hs.lcb0[gl]));
                }
            }
        }
        if (lateB && m >= 0) {
            if (!wait_smem_geq(&ha.mprog, (G + 1) * (k - 1) + (G - m), P.error, P.timeout_ns, lane)) return false;
            const uint32_t cb = valid ? wm.cbc[c][m] : 0u;
#pragma unroll
            for (int r = 0; r < T; ++r) acc[r] = max(acc[r], group_term<Q>(Rs, ha.lrf[1][r][m], cb));
        }
        poll_p();
    }
    if (t >= 1) {
        int leftv = 0;
        if (pt) {
            if (valid) leftv = (int)pt[c + 1][T - 1];
            __syncwarp();
            if (lane == 0) st_release_cta(&prodH->consumed, k);
        } else {
            // the left neighbour in another CTA: through its flag and global memory
            if (!warp_wait_geq(P.flags + sd.flag_off + I * NT + (J - 1), 1, P, lane)) return false;
            const int row = IT + 1 + c;
            if (valid && row <= JT - 1 && row < Np) leftv = ldcg16(Drow + (size_t)row * Np + (JT - 1));
            if (lateA) {
                uint32_t fa[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int ix = e * 32 + lane;
                    fa[e] = ix < T * G ? __ldcg(RF + (size_t)(IT + ix / G) * NG + (J - 1) * G + ix % G) : 0u;
                }
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int ix = e * 32 + lane;
                    memo_ensure<Q, kTwoVector, MEMO>(Rs, fa[e] & C::BMASK, ix < T * G, lane);
                    if (ix < T * G) ha.lrf[0][ix / G][ix % G] = group_word<Q>(fa[e]);
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    uint32_t fr[G];
                    if constexpr (G % 4 == 0) {
                        const uint4 *pv = reinterpret_cast<const uint4 *>(&ha.lrf[0][r][0]);
#pragma unroll
                        for (int v4 = 0; v4 < G / 4; ++v4) {
                            const uint4 w4 = pv[v4];
                            fr[4 * v4] = w4.x; fr[4 * v4 + 1] = w4.y; fr[4 * v4 + 2] = w4.z; fr[4 * v4 + 3] = w4.w;
                        }
                    } else {
#pragma unroll
                        for (int gl = 0; gl < G; ++gl) fr[gl] = ha.lrf[0][r][gl];
                    }
#pragma unroll
                    for (int gl = 0; gl < G; ++gl) acc[r] = max(acc[r], group_term<Q>(Rs, fr[gl], hs.lcb0[gl]));
                }
            }
        }
        if (valid) pp.left[c + 1] = (int16_t)leftv;
        if (c == 0) pp.left[0] = 0;
    }
    if (!p_done) {
        if (!warp_wait_geq(cntp, nfar, P, lane)) return false;
        merge_p();
    }
#pragma unroll
    for (int r = 0; r < T; ++r) pp.pm[r][c] = (int16_t)(acc[r] >> 16);
    __syncwarp();
    if (lane == 0) st_release_cta(&ha.prep_ready, k + 1);
    return true;
}

}  // namespace fold
