// fold_inst_tv9.cu -- instantiation of the persistent fold kernel (two-vector, q = 9).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv9(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<9, kTwoVector>(p, grid, st); }
int bps_tv9() { return blocks_per_sm_q<9, kTwoVector>(); }
size_t smem_tv9() { return smem_bytes_for<9, kTwoVector>(); }
}  // namespace fold
