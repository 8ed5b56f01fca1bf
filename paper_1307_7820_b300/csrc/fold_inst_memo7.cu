// fold_inst_memo7.cu -- instantiation of the persistent fold kernel, two-vector with the partially
// memoised table of Section 3.2 (q = 7).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_memo7(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<7, kTwoVector, true>(p, grid, st); }
}  // namespace fold
