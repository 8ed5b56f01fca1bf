// fold_inst_memo3.cu -- instantiation of the persistent fold kernel, two-vector with the partially
// memoised table of Section 3.2 (q = 3).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_memo3(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<3, kTwoVector, true>(p, grid, st); }
}  // namespace fold
