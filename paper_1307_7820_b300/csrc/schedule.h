// schedule.h -- ordered task list for the persistent fold kernel (host side).
#pragma once
#include <stddef.h>

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

// Same list for one sequence, with step_begin[t] = index of the first task of
// step t (the NEAR tasks of tile diagonal t and the chunks placed after them);
// step_begin[NT] = out.size().
void build_schedule_steps(int NT, int kc, int strip, std::vector<int4> &out, std::vector<int> &step_begin);

// Checks a single-sequence list (coverage, chunk counts, dependency order); 0 = valid.
int check_schedule(int NT, int kc, int strip, const std::vector<int4> &tasks);

}  // namespace fold
