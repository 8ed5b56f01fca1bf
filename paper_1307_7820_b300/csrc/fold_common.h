// fold_common.h -- internal layout and task definitions shared by the host
// scheduler and the CUDA kernels of libfold_b300 (not part of the public ABI).
//
// The DP table of one sequence (Section 2, Eq. 1) is padded to Np = NT*T
// positions (padding bases never pair) and cut into T x T tiles; tile (I,J)
// holds rows I*T.. and columns J*T.. .  T is a multiple of q, so tile borders
// are group borders: column group g covers columns g*q..g*q+q-1 and its row
// group covers rows g*q+1..g*q+q (Section 3.1).
#pragma once
#include <stdint.h>

namespace fold {

constexpr int kWarpsPerCta = 8;                 // warp-level workers per CTA
constexpr int kThreads = 32 * kWarpsPerCta;
constexpr int kColOff = 7;                      // Dcol offset: D(i,j) at Dcol[j*PC + i + 7]
constexpr int kRing = 8;                        // P (far partial max) ring depth in tile diagonals
constexpr int kNeg16 = -32768;                  // int16 "minus infinity" for the row closure
constexpr int kPadCode = 4;                     // padding base: pairs with nothing
constexpr int kTraceWords = 11;                 // 64-bit words per task trace record

// kSliding: Section 4's organisation with per-cell vectors; kFg: Section 3.2's FG algorithm (each its
// own per-column kernel, single folds only)
enum Method : int { kTwoVector = 0, kPlain = 1, kSliding = 2, kFg = 3 };
enum TaskType : int { kTaskNear = 0, kTaskFar = 1, kTaskFarStrip = 2 };

// tile edge for a given q (two-vector) or the plain kernel
__host__ __device__ constexpr int tile_of(int q, int method) {
    return method == kPlain ? 32 : q * (32 / q);
}
__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
// tiles per STRIP chunk: every lane of a strip chunk handles this many columns
// (two-vector: 4 while a tile has at most 4 groups, so the per-group column
// features of all 4 columns stay in registers; else 2)
__host__ __device__ constexpr int strip_of(int q, int method) {
    return method == kPlain ? 2 : (tile_of(q, method) / q <= 4 ? 4 : 2);
}

// Task word layout (int4): x = sequence index; y = type<<28 | I<<14 | J;
// NEAR: z = number of FAR chunks that feed the tile; FAR: z = Ka, w = Kb
// (inclusive tile-column range of the middle blocks).
__host__ __device__ inline int task_type(int y) { return (y >> 28) & 3; }
__host__ __device__ inline int task_I(int y) { return (y >> 14) & 0x3fff; }
__host__ __device__ inline int task_J(int y) { return y & 0x3fff; }
__host__ __device__ inline int task_pack(int type, int I, int J) { return (type << 28) | (I << 14) | J; }

// Per-sequence descriptor (device).  Offsets are in elements of the pools.
struct SeqDesc {
    int n;          // true length
    int NT;         // tiles per side
    int Np;         // NT*T
    int PC;         // column pitch of the column-major copy
    long long code_off;   // uint8 codes (Np entries, padding = kPadCode)
    long long drow_off;   // int16 row-major copy, Np*Np
    long long dcol_off;   // int16 column-major copy, Np*PC
    long long rf_off;     // uint32 row features, Np rows * (Np/q) groups
    long long cf_off;     // uint32 column features, (Np/q) groups * Np columns
    long long flag_off;   // int tile-done flags, NT*NT
    long long cnt_off;    // int far-chunk counters, NT*NT
    long long p_off;      // int P ring, kRing*NT*T*T
    int result_index;     // results[result_index] = D(0, n-1)
    int pad_;
};

struct FoldParams {
    const int4 *tasks;
    int ntasks;
    int *queue_head;          // next task index (tile tasks when the queues are split)
    // split queues: tasks[0, nnear) are the tile (NEAR) tasks and tasks[nnear, ntasks) the chunk
    // tasks, each part in list order; CTAs with blockIdx.x < near_ctas take only tile tasks (through
    // queue_head), the others only chunk tasks (through queue_head_far).  near_ctas == 0: one queue.
    int nnear;
    int near_ctas;
    int *queue_head_far;
    // column mode (split queues, one sequence): the tile tasks are not taken from the queue; warp w of
    // tile CTA b owns tile column b * cols_per_cta + w and computes its tiles bottom-up, (J,J) first.
    // tasks[0, nnear) still lists them (diagonal by diagonal) for their chunk counts.
    int col_mode;
    int cols_per_cta;
    // column mode, two-vector: warp w + kWarpsPerCta/2 of each tile CTA is the helper of column warp w
    // (cols_per_cta <= kWarpsPerCta/2): it prepares each tile's inputs and publishes each finished
    // tile, so the column warp only computes rows (see fold_column.cuh)
    int col_helpers;
    // column mode: the warps of a tile CTA whose columns are all finished take chunk tasks
    int col_join;
    // two-vector, q <= 9: launch the kernel instantiation in which R starts empty in each CTA and a
    // row R[h][*] is tabulated against every column vector the first time a warp of the CTA stages a
    // feature with horizontal vector h (Section 3.2's partially memoised variant); 0: the one that
    // copies the precomputed table in
    int memo;
    int *error;               // first error code (0 = none) and where
    const SeqDesc *seqs;
    const uint8_t *codes;
    int16_t *drow;
    int16_t *dcol;
    uint32_t *rf;
    uint32_t *cf;
    int *flags;
    int *cnt;
    int *pring;
    int *results;
    const uint8_t *rtab;      // R table in the kernel's smem layout
    unsigned long long pair64;  // bit (8x+y) = b(x,y)
    long long timeout_ns;     // bound on every device-side wait
    long long *trace;         // optional: kTraceWords words per task (see fold_trace_rec), or nullptr
    // serving ring (one persistent launch fed while it runs): ring_cap > 0 means task i is at
    // tasks[i % ring_cap] and exists once i < *ring_tail; the host advances *ring_tail (by copies, after
    // the tasks) and sets *ring_stop when it will publish no more; a worker whose claimed index is not
    // published waits (bounded) and leaves when the stop word is set.  Workers record the claimed
    // index in *ring_progress (host-mapped) every 256 claims, and answers go to host-mapped `results`
    // behind a system-scope fence.
    int ring_cap;
    const int *ring_tail;
    const int *ring_stop;
    int *ring_progress;
};

// error word values written by the kernel
enum KernelError : int { kErrNone = 0, kErrTimeout = 1, kErrBadTask = 2 };

}  // namespace fold
