// fold_inst_tv4.cu -- instantiation of the persistent fold kernel (two-vector, q = 4).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_tv4(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<4, kTwoVector>(p, grid, st); }
int bps_tv4() { return blocks_per_sm_q<4, kTwoVector>(); }
size_t smem_tv4() { return smem_bytes_for<4, kTwoVector>(); }
}  // namespace fold
