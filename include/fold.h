/*
 * fold.h -- C-ABI of libfold_b300: B300-native (sm_103a) Nussinov RNA folding
 * with the two-vector Four-Russians speedup of Venkatachalam, Gusfield and
 * Frid, "Faster Algorithms for RNA-folding using the Four-Russians method".
 *
 * What is computed (Section 2, Eq. 1).  For a sequence S of n bases the
 * library fills the table D(i,j), 0 <= i <= j < n, of the maximum number of
 * disjoint, non-crossing complementary base pairs inside S[i..j]:
 *     D(i,i) = D(i+1,i) = 0,
 *     D(i,j) = max( b(S_i,S_j) + D(i+1,j-1),  max_{i<k<=j} D(i,k-1) + D(k,j) ),
 * and the answer ("max pairs") D(0,n-1).  The default method evaluates the
 * second line with the two-vector scheme of Section 3.1: a table R over all
 * pairs of (q-1)-bit row/column difference vectors (built once by fold_init)
 * turns every group of q consecutive splits into one lookup (Eq. 3); splits
 * outside full groups are evaluated directly.  The plain method (kept as the
 * comparison) evaluates every split directly.  Both produce identical D.
 *
 * Conventions shared by every entry point:
 *   - positions are 0-based; bases are 'A','C','G','U' in either case, coded
 *     A=0, C=1, G=2, U=3; anything else is rejected with FOLD_EINVAL;
 *   - pair_mask bit (4*x + y) set means b(x,y) = 1, x being the base at the
 *     smaller position (asymmetric masks are allowed);
 *     FOLD_PAIRS_DEFAULT = {AU,UA,CG,GC,GU,UG}, FOLD_PAIRS_PAPER = {AU,UA,CG,GC};
 *   - no minimum hairpin loop: D(i,i+1) = b(S_i,S_{i+1});
 *   - 0 <= n <= FOLD_MAX_N; D values fit int16 (D <= n/2);
 *   - D tables handed back are n*n int16 row-major, D_out[i*n+j] = D(i,j) for
 *     i <= j and 0 for i > j;
 *   - every call returns a status code; no exception crosses the ABI;
 *   - the context owns its device state; the caller owns every buffer it
 *     passes, and inputs are not retained after a call returns (serve_submit
 *     copies the sequence);
 *   - a context is used by one thread at a time, except fold_serve_submit,
 *     fold_serve_poll and fold_serve_wait_any, which are thread-safe.
 */
#ifndef FOLD_B300_H
#define FOLD_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FOLD_ABI_VERSION 1
#define FOLD_MAX_N 65535
#define FOLD_PAIRS_DEFAULT ((uint16_t)0x5A48)
#define FOLD_PAIRS_PAPER ((uint16_t)0x1248)
#define FOLD_STATIC_MAX_N 1024

typedef struct fold_ctx fold_ctx;

enum fold_status {
    FOLD_OK = 0,
    FOLD_EINVAL = 1,    /* bad argument: q, mask, base letter, length, NULL pointer, size */
    FOLD_ENOMEM = 2,    /* device or host allocation failed, or workspace too small */
    FOLD_EAGAIN = 3,    /* serving: over the memory budget or the in-flight limit; retry later */
    FOLD_ETIMEOUT = 4,  /* a bounded device-side wait expired; results are not valid */
    FOLD_ECUDA = 5,     /* a CUDA runtime call failed */
    FOLD_ENOTREADY = 6  /* serving: the ticket is still in flight */
};

enum fold_method {
    FOLD_METHOD_TWO_VECTOR = 0, /* Section 3.1 / Section 4: R-table lookups per group of q splits */
    FOLD_METHOD_PLAIN = 1,      /* Section 2 / Section 4: every split evaluated (comparison kernel) */
    FOLD_METHOD_SLIDING = 2,    /* Section 4 as printed: one warp per column filling it bottom to top,
                                   groups of q splits relative to i and difference vectors stored at
                                   every cell (a second kernel organisation, kept for comparison).
                                   Single folds only (fold_score, fold_score_dev, fold_structure*);
                                   fold_batch, serving and the autotuner return FOLD_EINVAL.  Its
                                   workspace holds D plus two n*n uint32 vector tables (10*n^2 bytes). */
    FOLD_METHOD_FG = 3          /* Section 3.2's FG algorithm (Frid and Gusfield): Algorithm 1's groups,
                                   but a table per row and group, FG[i][g][c] = D(i,gq) + the best
                                   prefix of that row's vector against column vector c, built when the
                                   group completes (a comparison kernel in the per-column organisation).
                                   Single folds only, as FOLD_METHOD_SLIDING.  Its workspace holds D,
                                   the column vectors and n*(n/q+1)*2^(q-1) int16 table entries
                                   (about 1.2 GB at n = 6000, q = 8; 96 MB at q = 3). */
};

enum fold_option {
    FOLD_OPT_METHOD = 1,      /* fold_method; default FOLD_METHOD_TWO_VECTOR */
    FOLD_OPT_GRID = 2,        /* persistent CTAs; 0 = one wave (SM count x resident CTAs/SM) */
    FOLD_OPT_TIMEOUT_MS = 3,  /* bound on every device-side wait; default 5000 */
    FOLD_OPT_KCHUNK = 4,      /* middle tile columns per FAR chunk; 0 = automatic */
    FOLD_OPT_Q = 5,           /* read-only: q in use */
    FOLD_OPT_TILE = 6,        /* read-only: tile edge T of the current method */
    FOLD_OPT_LAUNCHES = 7,    /* read-only: kernels launched by this context so far */
    FOLD_OPT_TEST_DROP_TASK = 8, /* fault injection for tests: 1 = leave the tile (0,1) task out of the
                                    next single-sequence schedules, so its dependents' bounded waits
                                    expire and the call returns FOLD_ETIMEOUT; 0 = off (default) */
    FOLD_OPT_TIMING = 9,      /* 1 = record CUDA events around every persistent fold kernel launch */
    FOLD_OPT_KERNEL_NS = 10,  /* read-only: duration of the last timed fold kernel in ns (waits for it) */
    FOLD_OPT_TRACE = 11,      /* 1 = record per-task timestamps (see fold_trace_copy); 0 = off */
    FOLD_OPT_NEAR_CTAS = 12,  /* single folds: CTAs that run only tile tasks while the others run only
                                 middle-block chunks; -1 = automatic (default), 0 = one shared queue */
    FOLD_OPT_COLUMNS = 13,    /* with tile-only CTAs: each warp owns one tile column and computes it
                                 bottom-up (needs ceil(n_tiles / v) tile CTAs); -1 = automatic
                                 (default, v = 8), 0 = off, v = 1..8 = on, v columns per tile CTA */
    FOLD_OPT_BATCH_FLAT = 14, /* fold_batch's middle-block chunks: -1 = automatic / 1 = fixed size
                                 (FOLD_OPT_KCHUNK, default 64 blocks), 0 = the single fold's sizes
                                 (growing from both ends of each range) */
    FOLD_OPT_R_MEMO = 15,     /* Section 3.2's partially memoised variant (two-vector, q <= 9): 1 = each
                                 CTA starts with an empty R and tabulates the row R[h][*] against every
                                 column vector the first time one of its warps stages a horizontal
                                 vector h; 0 = the table precomputed at fold_init (default).  Results
                                 are identical; FOLD_EINVAL for q = 10, FOLD_EAGAIN while serving. */
    FOLD_OPT_BATCH_GATHER = 16, /* fold_batch's task list: 1 = gathered on the device from device copies of
                                 the per-size task templates, kept by the context (up to 1 GiB; only a
                                 segment list is copied per call; default); 0 = built on the host and
                                 copied whole.  Results are identical. */
    FOLD_OPT_COL_HELPERS = 17, /* single folds in column mode, two-vector: -1 = automatic (on where the
                                  layout has at most 4 columns per tile CTA and the fold at most 150
                                  tiles per side), 1 = on, 0 = off.  On, warp w + 4 of each tile CTA
                                  helps column warp w: it loads each next tile's inputs and does its
                                  late middle blocks' lookups and the chunk merge while the column warp
                                  computes rows.  Results are identical. */
    FOLD_OPT_SERVE_RING = 18,  /* serving: 1 (default) = requests in flight are folded by one persistent
                                  launch fed while it runs (a task ring the serving thread fills round
                                  by round); 0 = repeated launches, each a slice of tile diagonals of
                                  every request.  Set before fold_serve_start (FOLD_EAGAIN while
                                  serving).  Results are identical. */
    FOLD_OPT_COL_JOIN = 19,    /* single folds in column mode: -1 = automatic (on without column
                                  helpers), 1 = on, 0 = off.  On, the warps of a tile CTA whose tile
                                  columns are all finished take chunk tasks beside the chunk CTAs.
                                  Results are identical. */
    FOLD_OPT_SERVE_LONG_TILES = 20, /* serving: a request of at least this many tiles per side (32
                                  bases each) is long; default 160 (n >= 5089) */
    FOLD_OPT_SERVE_LONG_CAP = 21 /* serving: at most this many long requests in flight at once
                                  (default 2; 0 = no cap).  A long request beyond the cap waits, in
                                  arrival order among long ones, while shorter requests behind it
                                  are admitted past it (requests in flight share the device, so each
                                  long one admitted slows the others).  Both set before
                                  fold_serve_start (FOLD_EAGAIN while serving).  Results are
                                  identical. */
};

/* One record per task of the last traced persistent launch. */
typedef struct fold_trace_rec {
    int32_t worker;     /* global warp index that ran the task */
    int32_t task;       /* index in the ordered task list */
    int32_t type;       /* 0 = tile (NEAR), 1 = middle-block chunk (FAR) */
    int32_t I, J;       /* tile coordinates */
    int32_t seq;        /* sequence index within the launch */
    int32_t sm;         /* SM that ran the task (%smid) */
    int32_t reserved;   /* 0 */
    int64_t t_start;    /* %globaltimer ns when the worker took the task */
    int64_t t_deps;     /* ns when the tiles it reads were published */
    int64_t t_mid;      /* tile: ns when the partial max over middle blocks was complete;
                           chunk: ns when its lookups were done */
    int64_t t_end;      /* ns when its results were published */
    int64_t t_aux[3];   /* tile only: chunk partial maxima ready (0 if none), all rows done, stores issued */
} fold_trace_rec;

/* Creates a context on `device`.  q in [2,10] is the vector length of
 * Section 3.1 (0 picks the default, 8); pair_mask as above (must be non-zero
 * only on bits for codes 0..3).  Builds the R table (2^(2(q-1)) entries,
 * Section 3.1 preprocessing) on the device.  On success *out owns the context
 * (free with fold_destroy).  Errors: FOLD_EINVAL, FOLD_ECUDA, FOLD_ENOMEM. */
int fold_init(int q, uint16_t pair_mask, int device, fold_ctx **out);

/* Stops serving if active and releases every resource of the context. */
void fold_destroy(fold_ctx *ctx);

/* Static, human-readable text for a status code. */
const char *fold_strerror(int code);

/* Section 2's alphabet as the device entry points take it: writes the code of
 * seq[k] (A=0, C=1, G=2, U=3, either case) to codes_out[k] for k < n.  Both
 * buffers are host memory owned by the caller; codes_out needs n bytes.
 * FOLD_EINVAL if a letter is not one of ACGUacgu (codes_out is then partly
 * written), n is outside [0, FOLD_MAX_N] or a pointer is NULL with n > 0.
 * fold_score, fold_batch and fold_serve_submit apply the same mapping
 * themselves; callers of fold_score_dev, fold_structure_dev and
 * fold_score_static encode with this before copying the codes to the device. */
int fold_encode(const char *seq, int32_t n, uint8_t *codes_out);

/* Sets / reads an option (enum fold_option).  FOLD_EINVAL on an unknown
 * option or out-of-range value. */
int fold_set_option(fold_ctx *ctx, int option, int64_t value);
int fold_get_option(fold_ctx *ctx, int option, int64_t *value);

/* Copies up to `cap` trace records of the last traced launch (FOLD_OPT_TRACE)
 * into out and returns how many were written (or a negative status). */
int64_t fold_trace_copy(fold_ctx *ctx, fold_trace_rec *out, int64_t cap);

/* Host-only self-check of the task list the persistent kernel would run for
 * a single sequence of length n (no GPU needed): every middle block of every
 * tile is merged exactly once, each tile's chunk count is right, and every
 * task waits only on tasks placed before it, which is what makes the ordered
 * list deadlock-free (Section 4 wavefront, replaced by dependency flags).
 * kchunk = 0 picks the automatic chunk size.  Returns 0 if valid, a positive
 * failure code otherwise, or -FOLD_EINVAL for bad arguments (n above 65535,
 * or a tile count above 2048). */
int fold_schedule_check(int32_t n, int q, int method, int32_t kchunk);

/* Host-only check of the interleaved list fold_batch builds for `count`
 * sequences of lengths lens[] (fixed chunks of kchunk blocks, 0 = 64, as
 * fold_batch by default): every task carries a sequence index below count, and
 * each sequence's tasks appear exactly in the order of its single-sequence list,
 * which fold_schedule_check validates; so each sequence waits only on its own
 * earlier tasks; each distinct size's list is checked as by fold_schedule_check.
 * Returns 0 if valid, a positive failure code otherwise, or -FOLD_EINVAL for bad
 * arguments (a length above 65535 or a tile count above 512). */
int fold_batch_schedule_check(int32_t count, const int32_t *lens, int q, int method, int32_t kchunk);

/* Copies the R table to host memory: out[(h << (q-1)) | c] = R(h,c) for the
 * (q-1)-bit horizontal vector h and vertical vector c (bit p-1 holds
 * difference p; vertical differences stored as positive bits).  cap is the
 * size of out in bytes and must be >= 4^(q-1).  Section 3.1. */
int fold_rtable(fold_ctx *ctx, uint8_t *out, int64_t cap);

/* Folds one sequence from host memory (synchronous).  seq: n letters;
 * max_pairs (non-NULL) receives D(0,n-1) (0 for n <= 1); D_out (nullable)
 * receives the n*n table.  Device memory is managed by the context. */
int fold_score(fold_ctx *ctx, const char *seq, int32_t n, int32_t *max_pairs, int16_t *D_out);

/* Device-resident path for callers that own device memory (e.g. PyTorch).
 * fold_workspace_bytes returns the workspace size needed for length n (or a
 * negative status).  fold_score_dev enqueues the fold on `stream` (a
 * cudaStream_t; NULL is the CUDA default stream, as in the CUDA runtime API)
 * and returns without waiting:
 *   d_codes    n device bytes with codes 0..3 (not validated on the device);
 *   d_ws       device workspace of ws_bytes >= fold_workspace_bytes(ctx, n),
 *              256-byte aligned, owned by the caller, not reused until the
 *              stream has passed this call;
 *   d_max_pairs one device int32: D(0,n-1), or -FOLD_ETIMEOUT if a
 *              device-side wait expired;
 *   d_D_out    nullable device buffer of n*n int16 for the full table.
 * Inside the workspace D is kept twice as int16 (row-major and column-major,
 * padded to a multiple of the tile edge), plus the packed difference vectors
 * and the tile flags of the persistent kernel.
 * CUDA graphs: fold_score_dev may be recorded by stream capture (e.g. into a
 * torch.cuda.CUDAGraph) once one uncaptured call has folded that length with
 * the same options (it builds the task list, which needs allocations); a
 * replay then folds whatever the captured code buffers hold.  While a stream
 * is capturing, a length without a task list, FOLD_OPT_TIMING and
 * FOLD_OPT_TRACE return FOLD_EINVAL and nothing is recorded. */
int64_t fold_workspace_bytes(fold_ctx *ctx, int32_t n);
int fold_score_dev(fold_ctx *ctx, const uint8_t *d_codes, int32_t n, void *d_ws, int64_t ws_bytes,
                   int32_t *d_max_pairs, int16_t *d_D_out, void *stream);

/* Folds `count` sequences in one persistent launch (sequence-level and
 * wavefront parallelism together).  seqs[k] has lens[k] letters;
 * max_pairs_out[k] receives D_k(0,n_k-1); D_out may be NULL, and so may any
 * D_out[k] (else lens[k]*lens[k] int16).  Synchronous.  Returns FOLD_EINVAL
 * for a letter outside ACGU/acgu (nothing is folded).  The context keeps its
 * workspace, a pinned staging buffer and (FOLD_OPT_BATCH_GATHER) device copies
 * of the per-size task templates, up to 1 GiB, between calls; they are freed
 * by fold_destroy. */
int fold_batch(fold_ctx *ctx, int32_t count, const char *const *seqs, const int32_t *lens,
               int32_t *max_pairs_out, int16_t *const *D_out);

/* One optimal secondary structure (Section 2, traceback).  The paper stores
 * D*(i,j), the argmax of Eq. 1, beside D; here the argmax is re-evaluated from
 * the finished table at each cell the trace visits, by a one-block kernel, in a
 * fixed order of preference: base i unpaired if D(i,j) = D(i+1,j); else the
 * pair (i,j) if b(S_i,S_j) = 1 and D(i,j) = D(i+1,j-1) + 1; else the smallest
 * split k in [i+2, j] with D(i,j) = D(i,k-1) + D(k,j).  The structure has
 * D(0,n-1) pairs, no two of them cross, and every pair is allowed by the mask.
 * fold_structure: host string in (as fold_score); max_pairs out; partner_out
 *   (nullable, n int32): the base paired with each base or -1; dot_bracket_out
 *   (nullable, n+1 chars): '(' / ')' for the smaller / larger base of each
 *   pair, '.' otherwise, NUL-terminated.  Synchronous.
 * fold_structure_workspace_bytes / fold_structure_dev: the device-resident
 *   form (as fold_score_dev): d_ws of at least fold_structure_workspace_bytes(n)
 *   bytes, 256-byte aligned; d_max_pairs one int32 (-FOLD_ETIMEOUT if the fold
 *   failed, -FOLD_ECUDA if the trace found the table inconsistent); d_partner n
 *   int32.  Enqueued on `stream` (NULL = the default stream). */
int fold_structure(fold_ctx *ctx, const char *seq, int32_t n, int32_t *max_pairs, int32_t *partner_out,
                   char *dot_bracket_out);
int64_t fold_structure_workspace_bytes(fold_ctx *ctx, int32_t n);
int fold_structure_dev(fold_ctx *ctx, const uint8_t *d_codes, int32_t n, void *d_ws, int64_t ws_bytes,
                       int32_t *d_max_pairs, int32_t *d_partner, void *stream);

/* Autotuner.  The paper fixes q per run and has no rule for the GPU's launch
 * shapes, so they are measured.
 * fold_tune: for this context (its q and method) and length n, times every
 *   single-fold layout (one shared task queue; tile-only CTAs; column mode with
 *   4 or 8 columns per tile CTA) with three middle-block chunk sizes, `reps`
 *   timed folds each (1..100) after one warm-up, on a seeded synthetic uniform
 *   sequence of length n, all on the context's stream (synchronous).  The
 *   fastest is kept for n's size bucket (four per doubling) and used by later
 *   single folds of that size unless FOLD_OPT_NEAR_CTAS, FOLD_OPT_COLUMNS or
 *   FOLD_OPT_KCHUNK is set.  `out` receives the settings (as option values:
 *   near_ctas -1/0/k, columns -1/0/v, kchunk 0 = automatic), their time in ms,
 *   and the time of the automatic choice.  FOLD_EAGAIN while serving.
 * fold_tune_q: picks q in [q_min, q_max] (2..10) for pair_mask and method
 *   (0 two-vector, 1 plain: q 8 only) on `device`: with count == 1 it tunes a
 *   context per q for length lens[0]; with count > 1 it times fold_batch on a
 *   synthetic batch with lengths lens[0..count) (best of 3 wall-clock runs).
 *   `out` is the fastest q's result.  Creates and destroys its own contexts.
 * fold_tune_save / fold_tune_load: write / read the context's tuned entries
 *   to / from a text file, one line per entry, tagged with the device name, q
 *   and method; save keeps other tags' lines.  Load returns FOLD_EINVAL when
 *   the file has no entry for this device, q and method. */
typedef struct fold_tune_result {
    int32_t q;
    int32_t near_ctas;   /* FOLD_OPT_NEAR_CTAS value of the winner */
    int32_t columns;     /* FOLD_OPT_COLUMNS value of the winner */
    int32_t kchunk;      /* FOLD_OPT_KCHUNK value of the winner (0 = automatic) */
    float ms;            /* its fold time */
    float default_ms;    /* the automatic choice's fold time */
} fold_tune_result;
int fold_tune(fold_ctx *ctx, int32_t n, int32_t reps, fold_tune_result *out);
int fold_tune_q(int device, uint16_t pair_mask, int method, const int32_t *lens, int32_t count, int32_t q_min,
                int32_t q_max, fold_tune_result *out);
int fold_tune_save(fold_ctx *ctx, const char *path);
int fold_tune_load(fold_ctx *ctx, const char *path);

/* Allocation-free fold.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc when they fold -- code
 * running inside a framework whose own allocator must own all device memory,
 * services that allocate everything at start-up and must not allocate or
 * implicitly synchronise the device on the request path, plugins and
 * callbacks where allocation is not permitted.  It needs no context and no
 * workspace: its scratch is one fixed 8 MiB device array inside this library,
 * which every GPU that loads the library holds until the process exits.
 *   d_codes     n device bytes with codes 0..3;
 *   n           0 <= n <= FOLD_STATIC_MAX_N (1024), else FOLD_EINVAL;
 *   pair_mask   as for fold_init;
 *   d_max_pairs one device int32: D(0,n-1), or -FOLD_ETIMEOUT;
 *   d_D_out     nullable device buffer of n*n int16 for the full table;
 *   stream      cudaStream_t (NULL = the CUDA default stream); the call is
 *               enqueued there and returns without waiting.
 * Two-vector method with q = 8 on the current device.  It allocates no device
 * memory (no cudaMalloc, cudaFree or allocating library call).  All calls
 * share the one scratch array, which keeps the last call's contents (each
 * call clears what must start at zero), so calls that overlap on the GPU
 * (different streams or threads) race and corrupt each other: serialise
 * them.  The first call on a device does that device's set-up: it finds the
 * array's device address, builds the R table, copies the task lists of every
 * tile count up to FOLD_STATIC_MAX_N from host memory into the array and
 * synchronises the stream; make that first call before any stream capture.
 * Every later call does host arithmetic and enqueues one memset and a few
 * kernel launches, with no host-to-device copy (the sequence descriptor is
 * passed as a kernel argument).  The set-up is not redone after
 * cudaDeviceReset: do not use this entry point on a device after resetting it
 * in the same process. */
int fold_score_static(const uint8_t *d_codes, int32_t n, uint16_t pair_mask, int32_t *d_max_pairs,
                      int16_t *d_D_out, void *stream);

/* Measures the attainable rate of R-table lookups in shared memory (Section
 * 3.1, Eq. 3: a byte load at index (h << (q-1)) | c, an add and a max) with a
 * full GPU of resident warps on `device`.  mode 0: warp-uniform row h, lane
 * column c, indices in registers (the table-lookup pattern alone); mode 1:
 * the fold kernel's inner step (row-feature words staged in shared memory,
 * four per 16-byte broadcast load, the lane's column feature in a register);
 * mode 2: independent random (h, c) per lane (bank conflicts).  q in [2, 9]
 * (mode 0: [6, 9]); iters in [1, 2^20] steps of 32 lookups per thread.
 * Writes lookups per SM clock per SM (from each CTA's clock64 cycles) and,
 * if kernel_ms is not NULL, the timed launch's duration.  Allocates a few
 * bytes of device memory per call.  FOLD_EINVAL on bad arguments. */
int fold_lookup_rate(int device, int q, int mode, int32_t iters, double *lookups_per_clk_sm, double *kernel_ms);

/* A batch as one capturable launch.  fold_batch encodes host strings, builds
 * the task list and waits for the answers on every call; for a fixed set of
 * lengths fold_batch_plan_create does the host part once (synchronously; call
 * it before any stream capture): the sequences' workspace layout, the task
 * list of the one persistent launch (every sequence's Section 4 wavefront,
 * interleaved step by step as fold_batch does) and each sequence's offset in
 * the concatenated codes, all kept on the device by the plan.  The plan is
 * tied to ctx and to its q and method at creation (FOLD_EINVAL otherwise).
 * count >= 1 sequences; lens[k] in [0, FOLD_MAX_N]; sliding/FG methods:
 * FOLD_EINVAL.  fold_batch_plan_destroy synchronises the device first, so no
 * enqueued fold of the plan is still reading its lists. */
typedef struct fold_batch_plan fold_batch_plan;
int fold_batch_plan_create(fold_ctx *ctx, int32_t count, const int32_t *lens, fold_batch_plan **out);
/* Workspace bytes fold_batch_dev needs, and the bytes of its concatenated codes
 * (the sum of the lengths); negative status on a NULL plan. */
int64_t fold_batch_plan_workspace_bytes(const fold_batch_plan *plan);
int64_t fold_batch_plan_codes_bytes(const fold_batch_plan *plan);
void fold_batch_plan_destroy(fold_batch_plan *plan);
/* Enqueues the fold of the planned batch on `stream` (cudaStream_t, NULL =
 * the CUDA default stream) and returns without waiting:
 *   d_codes     device bytes, codes 0..3 of every sequence back to back:
 *               sequence k starts at lens[0] + ... + lens[k-1];
 *   d_ws        device workspace, >= fold_batch_plan_workspace_bytes, 256-byte
 *               aligned, caller-owned, not reused until the stream has passed
 *               this call (it also holds the tables, see fold_batch_dev_table);
 *   d_max_pairs count device int32: D(0, n_k - 1) (0 for n_k <= 1), or
 *               -FOLD_ETIMEOUT if a device-side wait expired.
 * It allocates nothing, copies nothing from the host and does not
 * synchronise: one memset and three kernel launches, which stream capture
 * records into a CUDA graph whose replays fold whatever d_codes then holds.
 * FOLD_EINVAL under capture with FOLD_OPT_TIMING or FOLD_OPT_TRACE on, or on a
 * bad argument; FOLD_ENOMEM if ws_bytes is too small. */
int fold_batch_dev(fold_ctx *ctx, const fold_batch_plan *plan, const uint8_t *d_codes, void *d_ws, int64_t ws_bytes,
                   int32_t *d_max_pairs, void *stream);
/* Enqueues the copy of sequence k's n_k x n_k int16 table (row-major, zero below
 * the diagonal) from the workspace of a fold_batch_dev call to device memory
 * d_D_out; nothing for n_k = 0.  Capturable like fold_batch_dev. */
int fold_batch_dev_table(fold_ctx *ctx, const fold_batch_plan *plan, const void *d_ws, int32_t k, int16_t *d_D_out,
                         void *stream);

/* Serving (continuous batching).  fold_serve_start starts a host scheduler
 * thread that admits submitted requests while the device memory their two
 * int16 D copies need (about 4*n^2 bytes each) fits `budget_bytes` and at
 * most `max_inflight` are in flight, of which at most FOLD_OPT_SERVE_LONG_CAP
 * are long (FOLD_OPT_SERVE_LONG_TILES; shorter requests are admitted past a
 * long one that waits for that cap).  A request arriving to an idle server
 * (n <= 8192) folds alone in one launch with the single fold's work split.
 * Otherwise the in-flight requests are folded by one persistent launch that
 * the thread feeds while it runs (FOLD_OPT_SERVE_RING, default): round after
 * round it publishes the next tile diagonal of every in-flight request into a
 * device task ring, so a request that arrives while others are on the GPU
 * joins at the next round, with no launch boundary to wait for; answers come
 * back through host-mapped memory, and the launch ends when nothing is in
 * flight.  While that launch runs it holds every SM: other kernels of the
 * process (folds on any context) start once the server is idle.  With
 * FOLD_OPT_SERVE_RING = 0 the requests are folded in repeated launches, each
 * advancing every in-flight request by a slice of tile diagonals.  Every warp
 * of a slice takes tile and chunk tasks from one queue, unless
 * FOLD_OPT_NEAR_CTAS was set above 0 when serving started (that many CTAs
 * then take only tile tasks).  fold_serve_submit copies the sequence and
 * returns a ticket (FOLD_EAGAIN if the request alone exceeds the budget or the
 * queue is full).  fold_serve_poll returns FOLD_ENOTREADY while in flight and
 * FOLD_OK once done, filling max_pairs (and D_out, n*n int16, if not NULL);
 * the ticket is then released.  fold_serve_stop drains nothing: in-flight
 * requests are abandoned and their tickets become invalid. */
int fold_serve_start(fold_ctx *ctx, int64_t budget_bytes, int32_t max_inflight);
int fold_serve_submit(fold_ctx *ctx, const char *seq, int32_t n, uint64_t *ticket);
int fold_serve_poll(fold_ctx *ctx, uint64_t ticket, int32_t *max_pairs, int16_t *D_out);
int fold_serve_stop(fold_ctx *ctx);

/* Blocks until a request has finished (done or failed) that this call has not
 * reported yet, for at most timeout_ms: FOLD_OK with its ticket (collect it with
 * fold_serve_poll), FOLD_ENOTREADY on timeout, FOLD_EINVAL if no serving loop
 * runs.  Tickets already collected by fold_serve_poll are skipped.  Every call
 * must have returned before fold_serve_stop. */
int fold_serve_wait_any(fold_ctx *ctx, int32_t timeout_ms, uint64_t *ticket);

/* Builds now, on up to 16 host threads, the task lists the serving loop (and
 * single folds) of this context use for every sequence length up to max_n:
 * they depend only on the length and are otherwise built when a length is
 * first seen, adding that time (up to about 10 ms at n = 8000) to the first
 * request of each size.  Lists are kept for the life of the process (up to
 * 512 MiB, least recently used dropped first).  It also copies to the device,
 * for lengths up to 8192, the list a request arriving to an idle server folds
 * with (about 240 MiB for all of them, kept with the context; otherwise made
 * at the first lone request of each size, about 1 ms at n = 8000); this
 * allocates device memory and may wait for work already on the device.
 * FOLD_EINVAL if ctx is NULL or max_n is outside [0, 65535]; FOLD_ECUDA if a
 * device copy failed. */
int fold_serve_warm(fold_ctx *ctx, int32_t max_n);

/* Counters of the serving loop since fold_serve_start (for monitoring and
 * tuning).  A "slice" is one persistent launch over the in-flight set. */
typedef struct fold_serve_stats {
    uint64_t slices;        /* persistent launches so far (lone requests, serving-ring launches, slices) */
    uint64_t tasks;         /* tasks those launches ran (on the ring: tasks published) */
    uint64_t admitted;      /* requests admitted into the device arena */
    uint64_t finished;      /* requests done or failed */
    double gpu_ms;          /* device time of the launches (CUDA events around each launch) */
    double slice_ms;        /* host wall time from a launch's first enqueue to its results on the host */
    double prep_ms;         /* host time gathering task lists, descriptors and (ring) copies */
    int32_t queued;         /* waiting for admission now */
    int32_t inflight;       /* on the device now */
    uint64_t solo;          /* requests that arrived to an idle server (nothing else in flight or
                               waiting, length <= 8192) and were folded in one launch with the
                               single-fold work split instead of slice by slice */
} fold_serve_stats;
/* FOLD_EINVAL if ctx or out is NULL or no serving loop runs. */
int fold_serve_stats_get(fold_ctx *ctx, fold_serve_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* FOLD_B300_H */
