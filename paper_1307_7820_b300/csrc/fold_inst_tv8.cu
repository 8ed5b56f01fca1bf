// fold_inst_tv8.cu -- instantiation of the persistent fold kernel (two-vector, q = 8).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv8(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<8, kTwoVector>(p, grid, st); }
int bps_tv8() { return blocks_per_sm_q<8, kTwoVector>(); }
size_t smem_tv8() { return smem_bytes_for<8, kTwoVector>(); }
}  // namespace fold
