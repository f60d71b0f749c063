// bisim_autotune: picks the degree-class thresholds and the hub chunk size of
// the dense round layout for the context's own graph by timing refinement
// rounds under each candidate. The partition never depends on these settings
// (every class computes the same exact signature); only the time does.
//
// Coordinate descent, one setting at a time, in this order:
//   mid_max_degree    rows above it take the hub path     (2048, 4096, 8192)
//   small_max_degree  rows up to it take one thread each  (8, 16, 32)
//   hub_chunk         edges per CTA on the hub path       (1024, 2048, 4096)
// Each candidate rebuilds the layout, runs one warm-up round and then times
// `rounds` rounds from P_0 with CUDA events on the caller's stream; the fastest
// value stays before the next setting is tuned. Batched contexts then tune
// batch_split (graphs up to it go to the persistent kernel, larger ones to the
// union's round kernels beside it) over (0, 2048, 8192, 32768, INT32_MAX), each
// candidate timed as a whole bisim_iterate of `rounds` rounds after a warm-up
// one.
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

bisim_status time_rounds(bisim_ctx* ctx, cudaStream_t s, int32_t rounds, float* out_ms) {
    ctx->dense_ready = false;
    bisim_status st;
    if ((st = dense_prepare(ctx, s)) != BISIM_OK) return st;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    int64_t blocks = 0;
    for (int pass = 0; pass < 2 && st == BISIM_OK; ++pass) {      // pass 0 warms up
        cudaMemcpyAsync(ctx->P[0], ctx->P0, sizeof(int32_t) * ctx->n, cudaMemcpyDeviceToDevice, s);
        dense_start(ctx, s);
        ctx->cur = 0;
        cudaEventRecord(a, s);
        for (int32_t r = 0; r < (pass == 0 ? 1 : rounds) && st == BISIM_OK; ++r) st = dense_round(ctx, s, &blocks);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *out_ms = ms;
    return st;
}

// One whole run of `rounds` rounds (batched contexts: both kernels), after a
// warm-up run.
bisim_status time_iterate(bisim_ctx* ctx, cudaStream_t s, int32_t rounds, float* out_ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    bisim_status st = BISIM_OK;
    for (int pass = 0; pass < 2 && st == BISIM_OK; ++pass) {
        int32_t r = 0, x = 0;
        int64_t blocks = 0;
        cudaEventRecord(a, s);
        st = run_rounds(ctx, rounds, 0, s, &r, &x, &blocks);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *out_ms = ms;
    return st;
}

}  // namespace

}  // namespace bisim

using namespace bisim;

extern "C" bisim_status bisim_autotune(bisim_ctx* ctx, int32_t rounds, bisim_options* out, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    if (rounds < 1 || rounds > 64) return set_error(ctx, BISIM_EINVAL, "rounds must be in [1, 64]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ctx->last_stream = stream;
    bisim_status st;
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK) return st;
    // candidates rebuild the layout from the vertex-ordered CSR
    if ((st = dense_prepare(ctx, s)) != BISIM_OK || (st = ensure_vertex_csr(ctx, s)) != BISIM_OK) return st;
    if (ctx->n > 0) {
        struct Setting {
            int32_t* field;
            int32_t candidates[3];
        };
        Setting settings[] = {{&ctx->opt.mid_max_degree, {2048, 4096, 8192}},
                              {&ctx->opt.small_max_degree, {8, 16, 32}},
                              {&ctx->opt.hub_chunk, {1024, 2048, 4096}}};
        for (Setting& set : settings) {
            const int32_t keep = *set.field;
            int32_t best = keep;
            float best_ms = FLT_MAX;
            for (int32_t c : set.candidates) {
                *set.field = c;
                float ms = 0.f;
                if ((st = time_rounds(ctx, s, rounds, &ms)) != BISIM_OK) {
                    *set.field = keep;
                    ctx->dense_ready = false;
                    return st;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            *set.field = best;
        }
        // the next bisim_iterate builds the layout with the chosen settings (the
        // incremental path buckets its frontiers with them on every batch)
        ctx->dense_ready = false;
        if (segment_usable(ctx)) {
            const int32_t keep = ctx->opt.batch_split;
            int32_t best = keep;
            float best_ms = FLT_MAX;
            for (int32_t c : {0, 2048, 8192, 32768, INT_MAX}) {
                ctx->opt.batch_split = c;
                float ms = 0.f;
                if ((st = time_iterate(ctx, s, rounds, &ms)) != BISIM_OK) {
                    ctx->opt.batch_split = keep;
                    return st;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            ctx->opt.batch_split = best;
        }
    }
    if (out) *out = ctx->opt;
    return BISIM_OK;
}
