// fold_inst_tv10.cu -- instantiation of the persistent fold kernel (two-vector, q = 10).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv10(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<10, kTwoVector>(p, grid, st); }
int bps_tv10() { return blocks_per_sm_q<10, kTwoVector>(); }
size_t smem_tv10() { return smem_bytes_for<10, kTwoVector>(); }
}  // namespace fold
