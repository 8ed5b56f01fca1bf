// fg.h -- Section 3.2's FG algorithm as a comparison kernel (host side).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fold {

struct FgParams {
    const uint8_t *codes;       // n codes 0..3
    int n;
    int ng;                     // groups per row: n/q + 1
    int16_t *drow;              // n*n, zeroed
    uint32_t *cv;               // n*ng column vectors (D(gq+1,j) << 16 | bits)
    int16_t *fgt;               // n*ng*2^(q-1) row-group tables
    int *progress;              // n counters: rows of each column done (zeroed)
    int *next_col;              // column counter (zeroed)
    int *error;                 // error word (zeroed)
    int *result;                // D(0, n-1)
    unsigned long long pair64;  // bit (8x+y) = b(x,y)
    long long timeout_ns;       // bound on every device-side wait
};

// Workspace of one fold: control | results | progress (zeroed) | codes | Drow | CV | FGT
struct FgLayout {
    int ng;
    size_t off_control, off_results, off_progress, zero_bytes, off_codes, off_drow, off_cv, off_fgt, bytes;
};

FgLayout fg_layout(int n, int q);
cudaError_t launch_fg(const FgParams &p, int q, int sm_count, cudaStream_t st);

}  // namespace fold
