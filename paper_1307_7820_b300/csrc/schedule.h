// schedule.h -- ordered task list for the persistent fold kernel (host side).
#pragma once
#include <stddef.h>

#include <memory>
#include <vector>
#include <vector_types.h>

namespace fold {

// Builds the task list for sequences with NTs[s] tiles per side; kc is the
// number of middle tile columns merged by one chunk (at most, with geometric
// sizes from the ends of each range; exactly, without); strip is the number of
// tiles a STRIP chunk covers (1 = no strips).
void build_schedule(const std::vector<int> &NTs, int kc, int strip, std::vector<int4> &out, bool geometric = true);
// The same list written to out[0, total) when cap >= total; returns total (out may be null to count).
size_t build_schedule_into(const std::vector<int> &NTs, int kc, int strip, bool geometric, int4 *out, size_t cap);

// The list of one sequence with NT tiles per side (sequence index 0 in every task), step by
// step: step t is tasks[near_begin[t], near_begin[t+1]), the NEAR tasks of tile diagonal t in
// [near_begin[t], chunk_begin[t]) and the chunks placed after them in the rest.
struct SeqTemplate {
    std::vector<int4> tasks;
    std::vector<int> near_begin, chunk_begin;
};
// Built once per (NT, kc, strip, geometric) and shared (process-wide, thread-safe cache).
std::shared_ptr<const SeqTemplate> seq_template(int NT, int kc, int strip, bool geometric);

// A batch's list as segments, in the order build_schedule_into writes it (for each step t, the
// NEAR tasks of tile diagonal t of every sequence, then every sequence's chunks placed at t):
// segment k is tasks [first, first + count) of template tpls[tpl], written with sequence index seq
// at position dst.  Returns the total number of tasks; tpls holds one template per distinct size.
struct ScheduleSeg {
    int tpl, first, count, seq;
    size_t dst;
};
size_t schedule_segments(const std::vector<int> &NTs, int kc, int strip, bool geometric,
                         std::vector<std::shared_ptr<const SeqTemplate>> &tpls, std::vector<ScheduleSeg> &segs);

// Checks a single-sequence list (coverage, chunk counts, dependency order); 0 = valid.
int check_schedule(int NT, int kc, int strip, const std::vector<int4> &tasks);

}  // namespace fold
