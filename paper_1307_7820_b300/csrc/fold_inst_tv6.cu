// fold_inst_tv6.cu -- instantiation of the persistent fold kernel (two-vector, q = 6).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv6(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<6, kTwoVector>(p, grid, st); }
int bps_tv6() { return blocks_per_sm_q<6, kTwoVector>(); }
size_t smem_tv6() { return smem_bytes_for<6, kTwoVector>(); }
}  // namespace fold
