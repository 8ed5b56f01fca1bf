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
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "fold_common.h"
#include "schedule.h"

namespace fold {

namespace {
struct Chunk { int type, I, J, Ka, Kb, step; };

// Splits [lo, hi] into chunks (appended to `out`, which is cleared first) whose sizes grow
// geometrically (1, 2, 4, ... up to kc) from both ends toward the middle.  The blocks at either
// end of a tile's middle range are the last to become ready (they need the most recent tiles),
// so they come in small pieces that finish quickly; the middle blocks, ready long before, form
// the big chunks.  Without `geometric` the chunks are kc blocks each (batches: the folds' own
// critical paths matter little there, the number of tasks does).
void split_range(int lo, int hi, int kc, bool geometric, std::vector<std::pair<int, int>> &out,
                 std::vector<std::pair<int, int>> &tail) {
    out.clear();
    tail.clear();
    if (!geometric) {
        for (int a = lo; a <= hi; a += kc) out.push_back({a, std::min(hi, a + kc - 1)});
        return;
    }
    int size = 1;
    while (lo <= hi) {
        const int a = std::min(size, hi - lo + 1);
        out.push_back({lo, lo + a - 1});
        lo += a;
        if (lo > hi) break;
        const int b = std::min(size, hi - lo + 1);
        tail.push_back({hi - b + 1, hi});
        hi -= b;
        size = std::min(2 * size, kc);
    }
    out.insert(out.end(), tail.rbegin(), tail.rend());
}

// The task list of one sequence (index 0), step by step.  Chunks are generated in order of
// (tile diagonal J-I, row I), a tile's single-tile chunks before the strip chunks starting at it,
// and then placed by a stable counting sort on their step: within a step the most urgent chunk
// (lowest diagonal, then row) comes first.
void build_one(int NT, int kc, int S, bool geometric, SeqTemplate &tp) {
    tp.tasks.clear();
    tp.near_begin.assign((size_t)NT + 1, 0);
    tp.chunk_begin.assign((size_t)std::max(NT, 0), 0);
    if (NT <= 0) return;
    std::vector<int> nfar((size_t)NT * NT, 0), per_step((size_t)NT, 0);
    std::vector<Chunk> chunks;
    std::vector<std::pair<int, int>> parts, tail;
    auto add = [&](int type, int I, int J, int Jl, int Ka, int Kb) {
        // placed right after the NEAR tasks of the diagonal that follows the last tile it reads
        // (and, past the P ring's depth, the tile whose P slot it reuses)
        int d = std::max(Kb - I, Jl - Ka);
        if (Jl - I >= kRing) d = std::max(d, Jl - I - kRing);
        chunks.push_back({type, I, J, Ka, Kb, d + 1});
        per_step[(size_t)d + 1]++;
        for (int Jt = J; Jt <= Jl; ++Jt) nfar[(size_t)I * NT + Jt]++;
    };
    for (int t = 4; t < NT; ++t) {
        for (int I = 0; I + t < NT; ++I) {
            const int J = I + t;
            // single-tile chunks: all middle blocks, or, where the tile is covered by a strip, the
            // blocks next to its two ends
            const int J0s = J / S * S;
            if (S > 1 && J0s - 2 >= I + S + 1) {
                // every block of either end range is last read from a tile on diagonal t-2 or
                // earlier and is needed by tile (I,J) alone: one chunk per range (fewer tasks, no
                // later than the last of its blocks)
                split_range(I + 2, I + S, kc, false, parts, tail);
                for (const auto &ck : parts) add(kTaskFar, I, J, J, ck.first, ck.second);
                split_range(J0s - 1, J - 2, kc, false, parts, tail);
                for (const auto &ck : parts) add(kTaskFar, I, J, J, ck.first, ck.second);
            } else {
                split_range(I + 2, J - 2, kc, geometric, parts, tail);
                for (const auto &ck : parts) add(kTaskFar, I, J, J, ck.first, ck.second);
            }
            // strip chunks over tiles (I, J..J+Seff-1), for strip starts J >= I+S+3
            if (S > 1 && J % S == 0 && J >= I + S + 3) {
                const int Jl = std::min(J + S - 1, NT - 1);
                split_range(I + S + 1, J - 2, kc, geometric, parts, tail);
                for (const auto &ck : parts) add(kTaskFarStrip, I, J, Jl, ck.first, ck.second);
            }
        }
    }
    // step t: NEAR tasks of tile diagonal t, then the chunks placed at t
    std::vector<size_t> slot((size_t)NT);
    size_t k = 0;
    for (int t = 0; t < NT; ++t) {
        tp.near_begin[(size_t)t] = (int)k;
        k += (size_t)(NT - t);
        tp.chunk_begin[(size_t)t] = (int)k;
        slot[(size_t)t] = k;
        k += (size_t)per_step[(size_t)t];
    }
    tp.near_begin[(size_t)NT] = (int)k;
    tp.tasks.resize(k);
    for (int t = 0; t < NT; ++t) {
        int4 *o = tp.tasks.data() + tp.near_begin[(size_t)t];
        for (int I = 0; I + t < NT; ++I) o[I] = make_int4(0, task_pack(kTaskNear, I, I + t), nfar[(size_t)I * NT + I + t], 0);
    }
    for (const Chunk &ck : chunks)
        tp.tasks[slot[(size_t)ck.step]++] = make_int4(0, task_pack(ck.type, ck.I, ck.J), ck.Ka, ck.Kb);
}

// Templates are kept for the life of the process (they depend only on the sizes), up to
// kTemplateCacheBytes of tasks; past that the least recently used ones no caller holds are
// dropped.
constexpr size_t kTemplateCacheBytes = size_t(512) << 20;
struct TemplateCache {
    std::mutex mu;
    std::map<std::tuple<int, int, int, bool>, std::pair<std::shared_ptr<const SeqTemplate>, unsigned long long>> m;
    size_t bytes = 0;
    unsigned long long clock = 0;
};
TemplateCache &template_cache() {
    static TemplateCache *c = new TemplateCache();   // never destroyed: used from threads that may outlive statics
    return *c;
}
size_t template_bytes(const SeqTemplate &t) { return t.tasks.size() * sizeof(int4); }
}  // namespace

std::shared_ptr<const SeqTemplate> seq_template(int NT, int kc, int strip, bool geometric) {
    if (kc < 1) kc = 1;
    if (strip < 1) strip = 1;
    const auto key = std::make_tuple(NT, kc, strip, geometric);
    TemplateCache &c = template_cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.m.find(key);
        if (it != c.m.end()) {
            it->second.second = ++c.clock;
            return it->second.first;
        }
    }
    auto tp = std::make_shared<SeqTemplate>();
    build_one(NT, kc, strip, geometric, *tp);
    std::lock_guard<std::mutex> lk(c.mu);
    auto ins = c.m.emplace(key, std::make_pair(std::shared_ptr<const SeqTemplate>(tp), ++c.clock));
    if (!ins.second) return ins.first->second.first;   // another thread built it meanwhile
    c.bytes += template_bytes(*tp);
    while (c.bytes > kTemplateCacheBytes) {
        auto victim = c.m.end();
        for (auto it = c.m.begin(); it != c.m.end(); ++it)
            if (it->second.first.use_count() == 1 && (victim == c.m.end() || it->second.second < victim->second.second))
                victim = it;
        if (victim == c.m.end()) break;
        c.bytes -= template_bytes(*victim->second.first);
        c.m.erase(victim);
    }
    return ins.first->second.first;
}

void build_schedule(const std::vector<int> &NTs, int kc, int strip, std::vector<int4> &out, bool geometric) {
    out.clear();
    out.resize(build_schedule_into(NTs, kc, strip, geometric, nullptr, 0));
    build_schedule_into(NTs, kc, strip, geometric, out.data(), out.size());
}

size_t schedule_segments(const std::vector<int> &NTs, int kc, int strip, bool geometric,
                         std::vector<std::shared_ptr<const SeqTemplate>> &tpls, std::vector<ScheduleSeg> &segs) {
    const int nseq = (int)NTs.size();
    int maxNT = 0;
    for (int v : NTs) maxNT = std::max(maxNT, v);
    // one template per distinct size (a batch has few)
    tpls.clear();
    segs.clear();
    std::map<int, int> index;
    std::vector<int> tix((size_t)nseq, -1);
    for (int q = 0; q < nseq; ++q) {
        const int v = NTs[q];
        if (v <= 0) continue;
        auto it = index.find(v);
        if (it == index.end()) {
            it = index.emplace(v, (int)tpls.size()).first;
            tpls.push_back(seq_template(v, kc, strip, geometric));
        }
        tix[(size_t)q] = it->second;
    }
    // within a step the sequences go longest first (a step's tasks depend only on earlier steps, so
    // any order there keeps the list valid): the longest chains get their tasks first, and the scan
    // of a step stops at the first sequence that has no tile diagonal t
    std::vector<int> ord;
    ord.reserve((size_t)nseq);
    for (int q = 0; q < nseq; ++q)
        if (tix[(size_t)q] >= 0) ord.push_back(q);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return NTs[a] > NTs[b]; });
    size_t k = 0;
    for (int t = 0; t < maxNT; ++t) {
        for (int part = 0; part < 2; ++part) {
            for (int q : ord) {
                if (t >= NTs[q]) break;
                const SeqTemplate *p = tpls[(size_t)tix[(size_t)q]].get();
                const int a = part == 0 ? p->near_begin[t] : p->chunk_begin[t];
                const int b = part == 0 ? p->chunk_begin[t] : p->near_begin[t + 1];
                if (b > a) segs.push_back({tix[(size_t)q], a, b - a, q, k});
                k += (size_t)(b - a);
            }
        }
    }
    return k;
}

size_t build_schedule_into(const std::vector<int> &NTs, int kc, int strip, bool geometric, int4 *out, size_t cap) {
    if (!out) {
        // the count alone: one template lookup per distinct size
        std::map<int, size_t> size_of;
        size_t total = 0;
        for (int v : NTs) {
            if (v <= 0) continue;
            auto it = size_of.find(v);
            if (it == size_of.end()) it = size_of.emplace(v, seq_template(v, kc, strip, geometric)->tasks.size()).first;
            total += it->second;
        }
        return total;
    }
    std::vector<std::shared_ptr<const SeqTemplate>> tpls;
    std::vector<ScheduleSeg> segs;
    const size_t total = schedule_segments(NTs, kc, strip, geometric, tpls, segs);
    if (cap < total) return total;
    auto copy = [&](size_t s0, size_t s1) {
        for (size_t g = s0; g < s1; ++g) {
            const ScheduleSeg &sg = segs[g];
            const int4 *src = tpls[(size_t)sg.tpl]->tasks.data() + sg.first;
            for (int e = 0; e < sg.count; ++e) {
                int4 v = src[e];
                v.x = sg.seq;
                out[sg.dst + (size_t)e] = v;
            }
        }
    };
    // copied by a few threads when the list is long: the segments split into ranges of about
    // equal task counts
    const unsigned hw = std::thread::hardware_concurrency();
    const int nth = total < (1u << 20) ? 1 : (int)std::max(1u, std::min(hw, 16u));
    if (nth == 1) {
        copy(0, segs.size());
    } else {
        std::vector<std::thread> th;
        size_t g = 0;
        for (int w = 0; w < nth && g < segs.size(); ++w) {
            const size_t want = total * (size_t)(w + 1) / (size_t)nth;
            size_t e = g;
            while (e < segs.size() && (w == nth - 1 || segs[e].dst < want)) ++e;
            if (e > g) th.emplace_back(copy, g, e);
            g = e;
        }
        if (g < segs.size()) copy(g, segs.size());
        for (auto &x : th) x.join();
    }
    return total;
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
