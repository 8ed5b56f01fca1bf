// schedule.h -- ordered task list for the persistent fold kernel (host side).
#pragma once
#include <vector>
#include <vector_types.h>

namespace fold {

// Builds the task list for sequences with NTs[s] tiles per side; kc is the
// number of middle tile columns merged by one FAR chunk.
void build_schedule(const std::vector<int> &NTs, int kc, std::vector<int4> &out);

}  // namespace fold
