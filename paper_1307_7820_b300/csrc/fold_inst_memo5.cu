// fold_inst_memo5.cu -- instantiation of the persistent fold kernel, two-vector with the partially
// memoised table of Section 3.2 (q = 5).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_memo5(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<5, kTwoVector, true>(p, grid, st); }
}  // namespace fold
