// fold_inst_tv5.cu -- instantiation of the persistent fold kernel (two-vector, q = 5).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv5(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<5, kTwoVector>(p, grid, st); }
int bps_tv5() { return blocks_per_sm_q<5, kTwoVector>(); }
size_t smem_tv5() { return smem_bytes_for<5, kTwoVector>(); }
}  // namespace fold
