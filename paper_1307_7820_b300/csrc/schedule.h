// schedule.h -- ordered task list for the persistent fold kernel (host side).
#pragma once
#include <vector>
#include <vector_types.h>

namespace fold {

// Builds the task list for sequences with NTs[s] tiles per side; kc is the
// number of middle tile columns merged by one FAR chunk.
void build_schedule(const std::vector<int> &NTs, int kc, std::vector<int4> &out);

// Same list for one sequence, with step_begin[t] = index of the first task of
// step t (the NEAR tasks of tile diagonal t and the chunks placed after them);
// step_begin[NT] = out.size().
void build_schedule_steps(int NT, int kc, std::vector<int4> &out, std::vector<int> &step_begin);

}  // namespace fold
