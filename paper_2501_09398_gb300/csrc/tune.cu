// Autotuner: time a list of (launch plan, iteration batch size) candidates
// on a context's own fields and pick the one that minimises the paper's
// total time T = T_C + T_E (Eq. 1) for a run of n_iters iterations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

using namespace gs;

namespace {

// Device copies of the fields a run modifies, so tuning leaves the context
// as it found it.
struct Snapshot {
    std::vector<void*> bufs;
    std::vector<int> ids;
    std::vector<size_t> bytes;
    int32_t parity = 0;
    int64_t time = 0;
};

size_t field_bytes(const gs_ctx* c, int id, int64_t pitch) {
    int64_t w, rows;
    ctx_shape(c, id, &w, &rows);
    return (size_t)pitch * rows * ctx_elem_bytes(c);
}

cudaError_t take(gs_ctx* c, Snapshot* s) {
    gs_get_parity(c, &s->parity);
    gs_get_time(c, &s->time);
    const bool heat = ctx_is_heat(c);
    std::vector<int> ids;
    if (heat) ids = {s->parity ? GS_FIELD_T1 : GS_FIELD_T0};
    else if (ctx_is_skel(c)) ids = {GS_FIELD_X};
    else ids = {GS_FIELD_EX, GS_FIELD_EY, GS_FIELD_EZ, GS_FIELD_HX, GS_FIELD_HY, GS_FIELD_HZ};
    cudaStream_t st = ctx_stream(c);
    for (int id : ids) {
        void* p;
        int64_t pitch;
        ctx_field(c, id, &p, &pitch);
        const size_t b = field_bytes(c, id, pitch);
        void* copy = nullptr;
        cudaError_t e = gs_malloc(&copy, b);
        if (e != cudaSuccess) return e;
        s->bufs.push_back(copy);
        s->ids.push_back(id);
        s->bytes.push_back(b);
        e = cudaMemcpyAsync(copy, p, b, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(st);
}

cudaError_t restore(gs_ctx* c, Snapshot* s) {
    cudaStream_t st = ctx_stream(c);
    cudaError_t err = cudaStreamSynchronize(st);
    gs_set_parity(c, s->parity);
    for (size_t k = 0; k < s->bufs.size() && err == cudaSuccess; ++k) {
        void* p;
        int64_t pitch;
        ctx_field(c, s->ids[k], &p, &pitch);
        err = cudaMemcpyAsync(p, s->bufs[k], s->bytes[k], cudaMemcpyDeviceToDevice, st);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    for (void* b : s->bufs) cudaFree(b);
    s->bufs.clear();
    if (!ctx_is_heat(c) && !ctx_is_skel(c)) gs_set_time(c, s->time);
    return err;
}

}  // namespace

extern "C" gs_status gs_autotune(gs_ctx* ctx, int64_t n_iters, int32_t reps, const gs_tune_candidate* cands,
                                 int32_t n_cands, gs_tune_result* results, int32_t* best_index) {
    if (!ctx || !cands || !results || n_cands < 1 || n_iters < 1 || reps < 1)
        return ctx_fail(ctx, GS_ERR_INVALID_ARG, "gs_autotune: NULL pointer, or n_cands/n_iters/reps < 1");
    {
        const bool heat = ctx_is_heat(ctx);
        const bool skel = ctx_is_skel(ctx);
        const int lo = heat ? GS_FIELD_T0 : (skel ? GS_FIELD_X : GS_FIELD_EX);
        const int hi = heat ? GS_FIELD_P : (skel ? GS_FIELD_X : GS_FIELD_HZ);
        for (int id = lo; id <= hi; ++id) {
            void* p;
            int64_t pitch;
            ctx_field(ctx, id, &p, &pitch);
            if (!p) return ctx_fail(ctx, GS_ERR_STATE, "gs_autotune: every field must be bound");
        }
    }
    gs_plan saved;
    gs_get_plan(ctx, &saved);
    Snapshot snap;
    cudaError_t e = take(ctx, &snap);
    if (e != cudaSuccess) {
        for (void* b : snap.bufs) cudaFree(b);
        return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                        std::string("gs_autotune snapshot: ") + cudaGetErrorString(e));
    }
    cudaStream_t st = ctx_stream(ctx);
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    double best_total = INFINITY;
    int32_t best = -1;
    gs_status fatal = GS_OK;
    for (int32_t i = 0; i < n_cands && fatal == GS_OK; ++i) {
        gs_tune_result& r = results[i];
        r.plan = cands[i].plan;
        r.batch_size = cands[i].batch_size;
        r.build_seconds = 0.0;
        r.exec_ms_per_iter = INFINITY;
        r.total_ms = INFINITY;
        gs_status rs = gs_set_plan(ctx, &cands[i].plan);
        r.status = rs;
        if (rs != GS_OK) continue;  // plan not runnable here: skipped
        gs_get_plan(ctx, &r.plan);
        const int64_t S = cands[i].batch_size;
        if (S < 0) {
            r.status = GS_ERR_INVALID_ARG;
            continue;
        }
        if (S > 0) {
            rs = gs_graph_build(ctx, S);
            r.status = rs;
            if (rs != GS_OK) {
                if (rs == GS_ERR_CUDA) fatal = rs;
                continue;
            }
            gs_stats s;
            gs_get_stats(ctx, &s);
            r.build_seconds = s.last_build_seconds;
        }
        // warm-up run (also builds any remainder graph), then timed runs
        rs = gs_step(ctx, n_iters, S);
        if (rs == GS_OK) rs = gs_sync(ctx);
        double best_ms = INFINITY;
        for (int32_t k = 0; k < reps && rs == GS_OK; ++k) {
            cudaEventRecord(ev0, st);
            rs = gs_step(ctx, n_iters, S);
            cudaEventRecord(ev1, st);
            if (rs != GS_OK) break;
            e = cudaEventSynchronize(ev1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (e != cudaSuccess) {
                fatal = ctx_fail(ctx, GS_ERR_CUDA, std::string("gs_autotune timing: ") + cudaGetErrorString(e));
                break;
            }
            best_ms = std::min(best_ms, (double)ms);
        }
        r.status = rs;
        if (rs != GS_OK) {
            if (rs == GS_ERR_CUDA) fatal = rs;
            continue;
        }
        r.exec_ms_per_iter = best_ms / (double)n_iters;
        r.total_ms = r.build_seconds * 1e3 + best_ms;
        if (r.total_ms < best_total) {
            best_total = r.total_ms;
            best = i;
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    gs_graph_destroy(ctx);
    gs_set_plan(ctx, &saved);
    e = restore(ctx, &snap);
    if (fatal != GS_OK) return fatal;
    if (e != cudaSuccess) return ctx_fail(ctx, GS_ERR_CUDA, std::string("gs_autotune restore: ") + cudaGetErrorString(e));
    if (best_index) *best_index = best;
    if (best < 0) return ctx_fail(ctx, GS_ERR_UNSUPPORTED, "gs_autotune: no candidate could run");
    return GS_OK;
}
