// fold_inst_plain.cu -- instantiation of the persistent fold kernel (plain Nussinov).
#include "fold_kernel.cuh"

namespace fold {
cudaError_t launch_plain(const FoldParams &p, int grid, cudaStream_t st) { return launch_q<8, kPlain>(p, grid, st); }
int bps_plain() { return blocks_per_sm_q<8, kPlain>(); }
size_t smem_plain() { return smem_bytes_for<8, kPlain>(); }
}  // namespace fold
