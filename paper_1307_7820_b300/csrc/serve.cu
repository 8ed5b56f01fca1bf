// serve.cu -- continuous-batching serving loop (placeholder until implemented).
#include "../../include/fold.h"
#include "api_internal.h"

extern "C" {
int fold_serve_start(fold_ctx *ctx, int64_t budget_bytes, int32_t max_inflight) {
    (void)ctx; (void)budget_bytes; (void)max_inflight;
    return FOLD_EINVAL;
}
int fold_serve_submit(fold_ctx *ctx, const char *seq, int32_t n, uint64_t *ticket) {
    (void)ctx; (void)seq; (void)n; (void)ticket;
    return FOLD_EINVAL;
}
int fold_serve_poll(fold_ctx *ctx, uint64_t ticket, int32_t *max_pairs, int16_t *D_out) {
    (void)ctx; (void)ticket; (void)max_pairs; (void)D_out;
    return FOLD_EINVAL;
}
int fold_serve_stop(fold_ctx *ctx) {
    (void)ctx;
    return FOLD_OK;
}
}
