// fold_inst_tv2.cu -- instantiation of the persistent fold kernel (two-vector, q = 2).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv2(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<2, kTwoVector>(p, grid, st); }
int bps_tv2() { return blocks_per_sm_q<2, kTwoVector>(); }
size_t smem_tv2() { return smem_bytes_for<2, kTwoVector>(); }
}  // namespace fold
