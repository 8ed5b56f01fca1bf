// schedule.cpp -- host-side builder of the ordered task list that the
// persistent fold kernel consumes (one atomic cursor, warp-level workers).
//
// Section 4 of the paper fills the table one diagonal at a time with a
// barrier per diagonal.  Here the unit is a T x T tile and the barrier is
// replaced by per-tile dependency flags:
//
//   NEAR(I,J)  computes tile (I,J) itself.  It waits for tiles (I,J-1) and
//              (I+1,J) (which by induction implies every tile to the left in
//              row I and below in column J), computes the two "late" middle
//              blocks K = I+1 and K = J-1 itself, waits until every FAR chunk
//              of the tile has been merged, and then runs the row-by-row
//              recurrence inside the tile.
//   FAR(I,J,Ka..Kb)  merges the Four-Russians group lookups of the middle
//              tile columns K in [Ka,Kb] (I+2 <= K <= J-2) into the tile's
//              partial maximum.  It needs tiles (I,Kb) and (Ka,J).
//
// A FAR chunk is placed right after the NEAR tasks of the tile diagonal
// that follows the last diagonal it depends on, so it is normally ready when
// a worker takes it and it runs while the critical NEAR chain advances.
// Every task depends only on tasks placed earlier in the list, and workers
// take tasks in list order, so the kernel can always make progress.
#include <algorithm>
#include <vector>

#include "fold_common.h"
#include "schedule.h"

namespace fold {

void build_schedule(const std::vector<int> &NTs, int kc, std::vector<int4> &out) {
    out.clear();
    int nseq = (int)NTs.size();
    int maxNT = 0;
    for (int v : NTs) maxNT = std::max(maxNT, v);
    if (kc < 1) kc = 1;
    // per sequence: chunks bucketed by placement step; NEAR tasks need their chunk counts
    struct Chunk { int I, J, Ka, Kb; };
    std::vector<std::vector<std::vector<Chunk>>> bucket(nseq);
    std::vector<std::vector<int>> nfar(nseq);
    for (int s = 0; s < nseq; ++s) {
        int NT = NTs[s];
        bucket[s].assign(NT > 0 ? NT : 1, {});
        nfar[s].assign((size_t)NT * NT, 0);
        for (int t = 4; t < NT; ++t) {
            for (int I = 0; I + t < NT; ++I) {
                int J = I + t;
                for (int Ka = I + 2; Ka <= J - 2; Ka += kc) {
                    int Kb = std::min(Ka + kc - 1, J - 2);
                    int d = std::max(Kb - I, J - Ka);
                    if (t >= kRing) d = std::max(d, t - kRing);
                    int place = d + 1;   // <= t-1 because Kb <= J-2 and Ka >= I+2
                    bucket[s][place].push_back({I, J, Ka, Kb});
                    nfar[s][(size_t)I * NT + J]++;
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
            int NT = NTs[s];
            if (t >= NT) continue;
            for (int I = 0; I + t < NT; ++I) {
                int J = I + t;
                out.push_back(make_int4(s, task_pack(kTaskNear, I, J), nfar[s][(size_t)I * NT + J], 0));
            }
        }
        for (int s = 0; s < nseq; ++s) {
            if (t >= NTs[s]) continue;
            for (const Chunk &c : bucket[s][t]) out.push_back(make_int4(s, task_pack(kTaskFar, c.I, c.J), c.Ka, c.Kb));
        }
    }
}

void build_schedule_steps(int NT, int kc, std::vector<int4> &out, std::vector<int> &step_begin) {
    std::vector<int> nts(1, NT);
    build_schedule(nts, kc, out);
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

}  // namespace fold
