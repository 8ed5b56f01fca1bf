// sliding.h -- Section 4's two-vector algorithm with per-cell difference vectors (host side).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fold {

struct SlidingParams {
    const uint8_t *codes;       // n codes 0..3
    int n;
    int16_t *drow;              // n*n, zeroed
    uint32_t *H;                // n*n horizontal vector words
    uint32_t *V;                // n*n vertical vector words (column-major)
    int *progress;              // n counters: rows of each column done (zeroed)
    int *next_col;              // column counter (zeroed)
    int *error;                 // error word (zeroed)
    int *result;                // D(0, n-1)
    const uint8_t *rtab;        // R table in the kernels' shared-memory layout
    unsigned long long pair64;  // bit (8x+y) = b(x,y)
    long long timeout_ns;       // bound on every device-side wait
};

// Workspace of one fold: control | results | progress (zeroed) | codes | Drow | H | V
struct SlidingLayout {
    size_t off_control, off_results, off_progress, zero_bytes, off_codes, off_drow, off_H, off_V, bytes;
};

SlidingLayout sliding_layout(int n);
cudaError_t launch_sliding(const SlidingParams &p, int q, int sm_count, cudaStream_t st);

}  // namespace fold
