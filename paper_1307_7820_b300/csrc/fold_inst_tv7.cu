// fold_inst_tv7.cu -- instantiation of the persistent fold kernel (two-vector, q = 7).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv7(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<7, kTwoVector>(p, grid, st); }
int bps_tv7() { return blocks_per_sm_q<7, kTwoVector>(); }
size_t smem_tv7() { return smem_bytes_for<7, kTwoVector>(); }
}  // namespace fold
