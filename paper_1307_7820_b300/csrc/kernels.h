// kernels.h -- host launchers for the kernels in fold_kernel.cu (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fold_common.h"

namespace fold {

size_t fold_smem_bytes(int q, int method);
int fold_blocks_per_sm(int q, int method);
// column mode with a helper warp per column (fold_column.cuh) exists for this q and method
bool fold_col_helpers_supported(int q, int method);
cudaError_t launch_finalize(const int *error, const int *results, int count, int32_t *out, cudaStream_t st);
cudaError_t launch_fold(const FoldParams &p, int q, int method, int grid, cudaStream_t st);
cudaError_t launch_rtable(int q, uint8_t *canon, uint8_t *packed, cudaStream_t st);
cudaError_t launch_extract(const int16_t *drow, int Np, int n, int16_t *out, cudaStream_t st);
// Section 2 traceback of a finished table (intervals traced in parallel); scratch:
// traceback_scratch_bytes(n) bytes, partner: n int32; *result becomes -fail_code on failure
size_t traceback_scratch_bytes(int n);
cudaError_t launch_traceback(const int16_t *drow, int Np, const uint8_t *codes, int n, unsigned long long pair64,
                             void *scratch, int32_t *partner, int32_t *result, int fail_code, long long timeout_ns,
                             int sm_count, cudaStream_t st);
cudaError_t launch_pad_codes(const uint8_t *in, int n, int Np, uint8_t *out, cudaStream_t st);
// out[segs[s].w + e] = store[segs[s].x + e] with .x = segs[s].z, for e < segs[s].y (a batch's task
// list gathered from device copies of its templates)
cudaError_t launch_gather_tasks(const int4 *store, const int4 *segs, int nseg, int4 *out, int sm_count,
                                cudaStream_t st);

}  // namespace fold
