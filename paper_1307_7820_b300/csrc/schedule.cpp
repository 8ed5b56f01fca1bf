// schedule.cpp -- host-side builder of the ordered task list that the
// persistent fold kernel consumes (one atomic cursor, warp-level workers).
//
// Section 4 of the paper fills the table one diagonal at a time with a
// barrier per diagonal.  Here the unit is a T x T tile and the barrier is
// replaced by per-tile dependency flags:
//
//   NEAR(I,J)  computes tile (I,J).  It waits for tiles (I,J-1) and (I+1,J)
//              (which by induction implies every tile to the left in row I
//              and below in column J), evaluates the two "late" middle blocks
//              K = I+1 and K = J-1 itself, waits until every chunk covering
//              the tile has been merged, and runs the row recurrence.
//   FAR(I,J,Ka..Kb)  merges the Four-Russians lookups of middle tile columns
//              K in [Ka,Kb] into the partial maximum of tile (I,J).
//   STRIP(I,J0,Ka..Kb)  the same for the S tiles (I,J0..J0+S-1) at once
//              (every lane handles S columns, so each broadcast row feature
//              serves S lookups).  A strip takes the middle blocks
//              K in [I+S+1, J0-2]; the few blocks next to each tile's own
//              diagonal (K in [I+2, I+S] and [J0-1, J-2]) stay in single-tile
//              chunks, so no tile waits on a chunk that needs a later tile.
//
// A chunk is placed right after the NEAR tasks of the tile diagonal that
// follows the last diagonal it depends on, so it is normally ready when a
// worker takes it and it runs while the critical NEAR chain advances.  Every
// task depends only on tasks placed earlier in the list, and workers take
// tasks in list order, so the kernel can always make progress.
#include <algorithm>
#include <vector>

#include "fold_common.h"
#include "schedule.h"

namespace fold {

namespace {
struct Chunk { int type, I, J, Ka, Kb; };

// Splits [lo, hi] into chunks whose sizes grow geometrically (1, 2, 4, ... up
// to kc) from both ends toward the middle.  The blocks at either end of a
// tile's middle range are the last to become ready (they need the most
// recent tiles), so they come in small pieces that finish quickly; the middle
// blocks, ready long before, form the big chunks.
std::vector<std::pair<int, int>> split_range(int lo, int hi, int kc) {
    std::vector<std::pair<int, int>> head, tail;
    int size = 1;
    while (lo <= hi) {
        const int a = std::min(size, hi - lo + 1);
        head.push_back({lo, lo + a - 1});
        lo += a;
        if (lo > hi) break;
        const int b = std::min(size, hi - lo + 1);
        tail.push_back({hi - b + 1, hi});
        hi -= b;
        size = std::min(2 * size, kc);
    }
    head.insert(head.end(), tail.rbegin(), tail.rend());
    return head;
}
}

void build_schedule(const std::vector<int> &NTs, int kc, int strip, std::vector<int4> &out) {
    out.clear();
    int nseq = (int)NTs.size();
    int maxNT = 0;
    for (int v : NTs) maxNT = std::max(maxNT, v);
    if (kc < 1) kc = 1;
    if (strip < 1) strip = 1;
    const int S = strip;
    std::vector<std::vector<std::vector<Chunk>>> bucket(nseq);
    std::vector<std::vector<int>> nfar(nseq);
    for (int s = 0; s < nseq; ++s) {
        const int NT = NTs[s];
        bucket[s].assign(NT > 0 ? NT : 1, {});
        nfar[s].assign((size_t)NT * NT, 0);
        auto place = [&](int d) { return d + 1; };
        // single-tile chunks
        for (int t = 4; t < NT; ++t) {
            for (int I = 0; I + t < NT; ++I) {
                const int J = I + t;
                const int J0 = J / S * S;
                const bool has_strip = S > 1 && J0 - 2 >= I + S + 1;
                int ranges[2][2] = {{I + 2, J - 2}, {1, 0}};
                if (has_strip) {
                    ranges[0][0] = I + 2; ranges[0][1] = I + S;
                    ranges[1][0] = J0 - 1; ranges[1][1] = J - 2;
                }
                for (auto &rg : ranges) {
                    for (const auto &ck : split_range(rg[0], rg[1], kc)) {
                        const int Ka = ck.first, Kb = ck.second;
                        int d = std::max(Kb - I, J - Ka);
                        if (t >= kRing) d = std::max(d, t - kRing);
                        bucket[s][place(d)].push_back({kTaskFar, I, J, Ka, Kb});
                        nfar[s][(size_t)I * NT + J]++;
                    }
                }
            }
        }
        // strip chunks over tiles (I, J0..J0+Seff-1)
        if (S > 1) {
            for (int I = 0; I < NT; ++I) {
                for (int J0 = (I + S + 3 + S - 1) / S * S; J0 < NT; J0 += S) {
                    const int Seff = std::min(S, NT - J0);
                    const int Jl = J0 + Seff - 1;
                    for (const auto &ck : split_range(I + S + 1, J0 - 2, kc)) {
                        const int Ka = ck.first, Kb = ck.second;
                        int d = std::max(Kb - I, Jl - Ka);
                        if (Jl - I >= kRing) d = std::max(d, Jl - I - kRing);
                        bucket[s][place(d)].push_back({kTaskFarStrip, I, J0, Ka, Kb});
                        for (int J = J0; J <= Jl; ++J) nfar[s][(size_t)I * NT + J]++;
                    }
                }
            }
        }
        // most urgent first: lower tile diagonal, then row
        for (auto &b : bucket[s])
            std::stable_sort(b.begin(), b.end(), [](const Chunk &a, const Chunk &c) {
                int da = a.J - a.I, dc = c.J - c.I;
                return da != dc ? da < dc : a.I < c.I;
            });
    }
    for (int t = 0; t < maxNT; ++t) {
        for (int s = 0; s < nseq; ++s) {
            const int NT = NTs[s];
            if (t >= NT) continue;
            for (int I = 0; I + t < NT; ++I) {
                const int J = I + t;
                out.push_back(make_int4(s, task_pack(kTaskNear, I, J), nfar[s][(size_t)I * NT + J], 0));
            }
        }
        for (int s = 0; s < nseq; ++s) {
            if (t >= NTs[s]) continue;
            for (const Chunk &c : bucket[s][t]) out.push_back(make_int4(s, task_pack(c.type, c.I, c.J), c.Ka, c.Kb));
        }
    }
}

void build_schedule_steps(int NT, int kc, int strip, std::vector<int4> &out, std::vector<int> &step_begin) {
    std::vector<int> nts(1, NT);
    build_schedule(nts, kc, strip, out);
    // tasks are emitted step by step: NEAR tasks of diagonal t, then the chunks placed at t
    step_begin.assign(NT + 1, (int)out.size());
    int t = -1;
    for (int k = 0; k < (int)out.size(); ++k) {
        if (task_type(out[k].y) == kTaskNear) {
            int d = task_J(out[k].y) - task_I(out[k].y);
            while (t < d) step_begin[++t] = k;
        }
    }
    step_begin[NT] = (int)out.size();
}

// Independent check of a single-sequence list: every middle block K of every
// tile (I,J) is covered exactly once, each tile's chunk count matches, and
// every task waits only on tasks placed before it.  Returns 0 or a code > 0.
int check_schedule(int NT, int kc, int strip, const std::vector<int4> &tasks) {
    const int S = strip < 1 ? 1 : strip;
    std::vector<int> pos((size_t)NT * NT, -1), cover((size_t)NT * NT * NT, 0), seen((size_t)NT * NT, 0);
    for (int k = 0; k < (int)tasks.size(); ++k)
        if (task_type(tasks[k].y) == kTaskNear) {
            const int I = task_I(tasks[k].y), J = task_J(tasks[k].y);
            if (I > J || J >= NT || pos[(size_t)I * NT + J] >= 0) return 1;
            pos[(size_t)I * NT + J] = k;
        }
    for (int I = 0; I < NT; ++I)
        for (int J = I; J < NT; ++J)
            if (pos[(size_t)I * NT + J] < 0) return 2;
    auto before = [&](int I, int J, int k) { return pos[(size_t)I * NT + J] < k; };
    for (int k = 0; k < (int)tasks.size(); ++k) {
        const int4 tk = tasks[k];
        const int ty = task_type(tk.y), I = task_I(tk.y), J = task_J(tk.y);
        if (ty == kTaskNear) {
            if (J > I && (!before(I, J - 1, k) || !before(I + 1, J, k))) return 3;
            continue;
        }
        const int Ka = tk.z, Kb = tk.w;
        const int Jl = ty == kTaskFarStrip ? std::min(J + S - 1, NT - 1) : J;
        if (Ka > Kb || Ka < I + 2 || Kb > J - 2) return 4;
        if (!before(I, Kb, k) || !before(Ka, Jl, k)) return 5;
        if (Jl - I >= kRing && !before(I, Jl - kRing, k)) return 6;
        for (int Jt = J; Jt <= Jl; ++Jt) {
            if (k > pos[(size_t)I * NT + Jt]) return 7;   // a chunk must precede the tile it feeds
            seen[(size_t)I * NT + Jt]++;
            for (int K = Ka; K <= Kb; ++K) cover[((size_t)I * NT + Jt) * NT + K]++;
        }
    }
    for (int I = 0; I < NT; ++I)
        for (int J = I; J < NT; ++J) {
            if (tasks[pos[(size_t)I * NT + J]].z != seen[(size_t)I * NT + J]) return 8;
            for (int K = 0; K < NT; ++K) {
                const int want = (K >= I + 2 && K <= J - 2) ? 1 : 0;
                if (cover[((size_t)I * NT + J) * NT + K] != want) return 9;
            }
        }
    (void)kc;
    return 0;
}

}  // namespace fold
