// tune.cu -- autotuner of the fold's launch settings.
//
// The paper fixes q per run and gives no rule for the GPU's tile, chunk or
// work-split shapes; their best values depend on n and on the device.  The
// tuner measures them instead of modelling them:
//
//   fold_tune      for one context (fixed q and method) and one length n: times
//                  the single-fold layouts (one shared task queue, tile-only
//                  CTAs, column mode with 4 or 8 columns per tile CTA) with
//                  three chunk sizes each on a seeded synthetic sequence, and
//                  keeps the fastest for n's size bucket (four buckets per
//                  doubling of n).  Later folds of that size use it unless an
//                  option forces a layout.
//   fold_tune_q    picks q: one context per q in a range, each tuned (single
//                  length) or timed on a batch of the given lengths.
//   fold_tune_save / fold_tune_load   keep the per-size settings in a text file
//                  (one line per entry, tagged with the device name, q and method).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/fold.h"
#include "api_internal.h"
#include "fold_common.h"

namespace fold {
namespace {

// splitmix64: the seeded uniform ACGU input of the timing runs
uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
std::string synthetic_sequence(int n, uint64_t seed) {
    static const char kBases[4] = {'A', 'C', 'G', 'U'};
    std::string s((size_t)n, 'A');
    for (int k = 0; k < n; ++k) s[(size_t)k] = kBases[splitmix64(seed) & 3];
    return s;
}

struct Saved {
    int near_opt, cols_opt, kc;
};
Saved save_opts(const fold_ctx *ctx) { return {ctx->near_ctas_opt, ctx->columns_opt, ctx->kc_override}; }
void restore_opts(fold_ctx *ctx, const Saved &s) {
    ctx->near_ctas_opt = s.near_opt;
    ctx->columns_opt = s.cols_opt;
    ctx->kc_override = s.kc;
}

std::string device_name(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    std::string s = prop.name;
    std::replace(s.begin(), s.end(), ' ', '_');
    return s;
}

}  // namespace
}  // namespace fold

using namespace fold;

extern "C" {

int fold_tune(fold_ctx *ctx, int32_t n, int32_t reps, fold_tune_result *out) {
    if (!ctx || !out || n < 1 || n > FOLD_MAX_N || reps < 1 || reps > 100 || ctx->method >= kSliding) return FOLD_EINVAL;
    if (ctx->serve) return FOLD_EAGAIN;   // the serving thread owns the context's stream
    cudaSetDevice(ctx->device);
    memset(out, 0, sizeof *out);
    out->q = ctx->q;
    out->near_ctas = -1;
    out->columns = -1;

    const int64_t wsb = fold_workspace_bytes(ctx, n);
    if (wsb <= 0) return FOLD_EINVAL;
    const std::string seq = synthetic_sequence(n, 0x5EEDull + (uint64_t)n);
    std::vector<uint8_t> codes((size_t)n);
    for (int k = 0; k < n; ++k) codes[(size_t)k] = (uint8_t)(strchr("ACGU", seq[(size_t)k]) - "ACGU");
    uint8_t *d_codes = nullptr, *d_ws = nullptr;
    int32_t *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FOLD_OK;
    if (cudaMalloc(&d_codes, (size_t)n) != cudaSuccess || cudaMalloc(&d_ws, (size_t)wsb) != cudaSuccess ||
        cudaMalloc(&d_out, sizeof(int32_t)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rc = FOLD_ENOMEM;
    }
    if (rc == FOLD_OK && cudaMemcpy(d_codes, codes.data(), (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = FOLD_ECUDA;

    const Saved saved = save_opts(ctx);
    const int T = tile_of(ctx->q, ctx->method);
    const int NT = (n + T - 1) / T;
    const int grid = grid_for(ctx);
    const int kc0 = kc_auto(NT);
    struct Cand {
        int near_opt, cols_opt;
    };
    std::vector<Cand> layouts = {{-1, -1}, {0, -1}};   // automatic (the cost model) first, then one queue
    if (NT >= 2) {
        const int k8 = std::max(2, std::min((NT + kWarpsPerCta - 1) / kWarpsPerCta, grid / 6));
        layouts.push_back({std::min(k8, grid - 1), 0});
        for (int cpc : {4, 8})
            if ((NT + cpc - 1) / cpc <= grid - 1) layouts.push_back({-1, cpc});
    }
    std::vector<int> kcs = {kc0};
    if (kc0 / 2 >= 1 && kc0 / 2 != kc0) kcs.push_back(kc0 / 2);
    if (std::min(64, kc0 * 2) != kc0) kcs.push_back(std::min(64, kc0 * 2));

    float best = 1e30f, def = 0.f;
    TuneEntry best_e;
    int32_t ref_score = -1;
    for (const Cand &cd : layouts) {
        for (int kc : kcs) {
            if (rc != FOLD_OK) break;
            if (cd.near_opt == -1 && cd.cols_opt == -1 && kc != kc0) continue;   // the default once
            ctx->near_ctas_opt = cd.near_opt;
            ctx->columns_opt = cd.cols_opt;
            ctx->kc_override = kc == kc0 ? 0 : kc;
            float tmin = 1e30f;
            for (int r = 0; r <= reps && rc == FOLD_OK; ++r) {   // one warm-up launch, then reps timed
                if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) rc = FOLD_ECUDA;
                if (rc == FOLD_OK) rc = enqueue_single(ctx, d_codes, n, d_ws, (size_t)wsb, d_out, nullptr, ctx->stream);
                if (rc == FOLD_OK && cudaEventRecord(e1, ctx->stream) != cudaSuccess) rc = FOLD_ECUDA;
                if (rc == FOLD_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = FOLD_ECUDA;
                float ms = 0.f;
                if (rc == FOLD_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = FOLD_ECUDA;
                if (rc == FOLD_OK && r > 0) tmin = std::min(tmin, ms);
            }
            int32_t score = 0;
            if (rc == FOLD_OK && cudaMemcpy(&score, d_out, sizeof score, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = FOLD_ECUDA;
            if (rc == FOLD_OK && score < 0) rc = -score;   // a device wait failed (-status)
            if (rc == FOLD_OK && ref_score >= 0 && score != ref_score) rc = FOLD_ECUDA;   // layouts disagree
            if (rc != FOLD_OK) break;
            ref_score = score;
            if (cd.near_opt == -1 && cd.cols_opt == -1) def = tmin;
            if (tmin < best) {
                best = tmin;
                best_e.near_opt = cd.near_opt;
                best_e.cols_opt = cd.cols_opt;
                best_e.kc = kc == kc0 ? 0 : kc;
                best_e.ms = tmin;
            }
        }
    }
    restore_opts(ctx, saved);
    if (rc == FOLD_OK) {
        ctx->tune[tune_bucket(n)] = best_e;
        out->near_ctas = best_e.near_opt;
        out->columns = best_e.cols_opt;
        out->kchunk = best_e.kc;
        out->ms = best;
        out->default_ms = def;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_codes);
    cudaFree(d_ws);
    cudaFree(d_out);
    return rc;
}

int fold_tune_q(int device, uint16_t pair_mask, int method, const int32_t *lens, int32_t count, int32_t q_min,
                int32_t q_max, fold_tune_result *out) {
    if (!out || !lens || count < 1 || q_min < 2 || q_max > 10 || q_min > q_max) return FOLD_EINVAL;
    if (method != 0 && method != 1) return FOLD_EINVAL;
    for (int32_t k = 0; k < count; ++k)
        if (lens[k] < 0 || lens[k] > FOLD_MAX_N) return FOLD_EINVAL;
    memset(out, 0, sizeof *out);
    out->ms = 1e30f;
    // synthetic batch with the given lengths (also the single-length case)
    std::vector<std::string> seqs((size_t)count);
    std::vector<const char *> ptrs((size_t)count);
    for (int32_t k = 0; k < count; ++k) {
        seqs[(size_t)k] = synthetic_sequence(lens[k], 0xBA7Cull + (uint64_t)k);
        ptrs[(size_t)k] = seqs[(size_t)k].c_str();
    }
    std::vector<int32_t> res((size_t)count);
    int found = 0;
    for (int q = q_min; q <= q_max; ++q) {
        if (method == 1 && q != 8) continue;   // the plain kernel has no q
        fold_ctx *ctx = nullptr;
        int rc = fold_init(q, pair_mask, device, &ctx);
        if (rc != FOLD_OK) return rc;
        rc = fold_set_option(ctx, FOLD_OPT_METHOD, method);
        fold_tune_result r;
        memset(&r, 0, sizeof r);
        r.q = q;
        if (rc == FOLD_OK && count == 1) {
            rc = fold_tune(ctx, lens[0], 3, &r);
        } else if (rc == FOLD_OK) {
            // batch: one warm-up, then the best of three wall-clock runs of the whole call
            rc = fold_batch(ctx, count, ptrs.data(), lens, res.data(), nullptr);
            double tmin = 1e30;
            for (int rep = 0; rep < 3 && rc == FOLD_OK; ++rep) {
                const auto t0 = std::chrono::steady_clock::now();
                rc = fold_batch(ctx, count, ptrs.data(), lens, res.data(), nullptr);
                const auto t1 = std::chrono::steady_clock::now();
                tmin = std::min(tmin, std::chrono::duration<double, std::milli>(t1 - t0).count());
            }
            r.ms = (float)tmin;
            r.default_ms = (float)tmin;
        }
        fold_destroy(ctx);
        if (rc != FOLD_OK) return rc;
        if (r.ms < out->ms) {
            *out = r;
            found = 1;
        }
    }
    return found ? FOLD_OK : FOLD_EINVAL;
}

int fold_tune_save(fold_ctx *ctx, const char *path) {
    if (!ctx || !path) return FOLD_EINVAL;
    // keep other contexts' lines, replace this one's
    const std::string tag = device_name(ctx->device) + " q=" + std::to_string(ctx->q) + " method=" + std::to_string(ctx->method);
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof line, f)) {
            std::string s(line);
            if (s.rfind("fold-tune-v1 ", 0) == 0 && s.find(" " + tag + " ") != std::string::npos) continue;
            keep.push_back(s);
        }
        fclose(f);
    }
    FILE *f = fopen(path, "w");
    if (!f) return FOLD_EINVAL;
    for (const std::string &s : keep) fputs(s.c_str(), f);
    for (const auto &kv : ctx->tune)
        fprintf(f, "fold-tune-v1 %s bucket=%d near=%d cols=%d kc=%d ms=%.4f\n", tag.c_str(), kv.first,
                kv.second.near_opt, kv.second.cols_opt, kv.second.kc, (double)kv.second.ms);
    const int bad = ferror(f);
    fclose(f);
    return bad ? FOLD_EINVAL : FOLD_OK;
}

int fold_tune_load(fold_ctx *ctx, const char *path) {
    if (!ctx || !path) return FOLD_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return FOLD_EINVAL;
    const std::string dev = device_name(ctx->device);
    char line[512];
    int loaded = 0;
    while (fgets(line, sizeof line, f)) {
        char name[256];
        int q = 0, method = 0, bucket = 0, near_opt = 0, cols_opt = 0, kc = 0;
        float ms = 0.f;
        if (sscanf(line, "fold-tune-v1 %255s q=%d method=%d bucket=%d near=%d cols=%d kc=%d ms=%f", name, &q, &method,
                   &bucket, &near_opt, &cols_opt, &kc, &ms) != 8)
            continue;
        if (dev != name || q != ctx->q || method != ctx->method) continue;
        if (near_opt < -1 || near_opt > 4096 || cols_opt < -1 || cols_opt > kWarpsPerCta || kc < 0 || kc > 64) continue;
        TuneEntry e;
        e.near_opt = near_opt;
        e.cols_opt = cols_opt;
        e.kc = kc;
        e.ms = ms;
        ctx->tune[bucket] = e;
        ++loaded;
    }
    fclose(f);
    return loaded > 0 ? FOLD_OK : FOLD_EINVAL;
}

}  // extern "C"
