// fold_inst_tv3.cu -- instantiation of the persistent fold kernel (two-vector, q = 3).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv3(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<3, kTwoVector>(p, grid, st); }
int bps_tv3() { return blocks_per_sm_q<3, kTwoVector>(); }
size_t smem_tv3() { return smem_bytes_for<3, kTwoVector>(); }
}  // namespace fold
