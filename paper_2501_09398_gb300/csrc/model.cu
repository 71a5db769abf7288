// The paper's analytic performance model (Sec. III-B) and the batch-size
// choice it implies.
//   T   = T_C + T_E                      (Eq. 1)
//   T_C = k_c S + b_c                    (Eq. 2, graph creation incl. upload)
//   T_E = a / S + b                      (Eq. 6; a = I_k (T_a - T_i),
//                                         b = I_k (T_k + T_i) - T_a + T_l)
// Fits are ordinary least squares on measured (S, T_C) and (S, T_E) pairs;
// the chosen S minimises Eq. 1 over the admissible sizes.  Host code only.
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

using namespace gs;

namespace {

// Least squares y = p*u + q over n points; false if u is constant.
bool line_fit(const double* u, const double* y, int n, double* p, double* q) {
    double su = 0, sy = 0;
    for (int i = 0; i < n; ++i) {
        su += u[i];
        sy += y[i];
    }
    const double mu = su / n, my = sy / n;
    double suu = 0, suy = 0;
    for (int i = 0; i < n; ++i) {
        suu += (u[i] - mu) * (u[i] - mu);
        suy += (u[i] - mu) * (y[i] - my);
    }
    if (!(suu > 0)) return false;
    *p = suy / suu;
    *q = my - *p * mu;
    return true;
}

bool all_finite(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

extern "C" {

gs_status gs_model_fit(const double* S, const double* t_create, const double* t_exec, int32_t n, gs_model* out) {
    if (!S || !t_create || !t_exec || !out || n < 2) return global_fail(GS_ERR_INVALID_ARG, "gs_model_fit: need >= 2 points");
    for (int i = 0; i < n; ++i)
        if (!(S[i] >= 1)) return global_fail(GS_ERR_INVALID_ARG, "gs_model_fit: batch sizes must be >= 1");
    if (!all_finite(t_create, n) || !all_finite(t_exec, n)) return global_fail(GS_ERR_NUMERIC, "gs_model_fit: non-finite time");
    std::vector<double> inv(n);
    for (int i = 0; i < n; ++i) inv[i] = 1.0 / S[i];
    gs_model m{};
    if (!line_fit(S, t_create, n, &m.k_c, &m.b_c) || !line_fit(inv.data(), t_exec, n, &m.a, &m.b))
        return global_fail(GS_ERR_INVALID_ARG, "gs_model_fit: batch sizes must not all be equal");
    double ec = 0, ee = 0;
    for (int i = 0; i < n; ++i) {
        ec += std::fabs(m.k_c * S[i] + m.b_c - t_create[i]);
        ee += std::fabs(m.a * inv[i] + m.b - t_exec[i]);
    }
    m.mae_create = ec / n;
    m.mae_exec = ee / n;
    *out = m;
    return GS_OK;
}

gs_status gs_model_total(const gs_model* m, double S, double* total_out) {
    if (!m || !total_out || !(S >= 1))
        return global_fail(GS_ERR_INVALID_ARG, "gs_model_total: need a model, an output and S >= 1");
    *total_out = m->k_c * S + m->b_c + m->a / S + m->b;
    return GS_OK;
}

gs_status gs_model_pick(const gs_model* m, const int64_t* cands, int32_t n, int64_t* best_S, double* best_T) {
    if (!m || !cands || n < 1 || !best_S) return global_fail(GS_ERR_INVALID_ARG, "gs_model_pick: bad arguments");
    double bt = INFINITY;
    int64_t bs = 0;
    for (int i = 0; i < n; ++i) {
        if (cands[i] < 1) return global_fail(GS_ERR_INVALID_ARG, "gs_model_pick: candidates must be >= 1");
        const double t = m->k_c * (double)cands[i] + m->b_c + m->a / (double)cands[i] + m->b;
        if (t < bt || (t == bt && cands[i] < bs)) {
            bt = t;
            bs = cands[i];
        }
    }
    *best_S = bs;
    if (best_T) *best_T = bt;
    return GS_OK;
}

gs_status gs_model_calibrate(gs_ctx* ctx, int64_t n_iters, const int64_t* S_list, int32_t n, int32_t reps,
                             gs_model* out) {
    if (!ctx || !S_list || n < 2 || n_iters < 1 || reps < 1 || !out)
        return ctx_fail(ctx, GS_ERR_INVALID_ARG, "gs_model_calibrate: need >= 2 batch sizes, n_iters, reps >= 1");
    gs_plan plan;
    gs_get_plan(ctx, &plan);
    std::vector<gs_tune_candidate> c(n);
    for (int i = 0; i < n; ++i) {
        if (S_list[i] < 1) return ctx_fail(ctx, GS_ERR_INVALID_ARG, "gs_model_calibrate: batch sizes must be >= 1");
        c[i].plan = plan;
        c[i].batch_size = S_list[i];
    }
    std::vector<gs_tune_result> r(n);
    int32_t best = -1;
    gs_status st = gs_autotune(ctx, n_iters, reps, c.data(), n, r.data(), &best);
    if (st != GS_OK) return st;
    std::vector<double> s(n), tc(n), te(n);
    for (int i = 0; i < n; ++i) {
        if (r[i].status != GS_OK) return ctx_fail(ctx, (gs_status)r[i].status, "gs_model_calibrate: a run failed");
        s[i] = (double)S_list[i];
        tc[i] = r[i].build_seconds;
        te[i] = r[i].exec_ms_per_iter * 1e-3 * (double)n_iters;
    }
    st = gs_model_fit(s.data(), tc.data(), te.data(), n, out);
    if (st != GS_OK) return ctx_fail(ctx, st, gs_last_error(nullptr));
    return GS_OK;
}

gs_status gs_pick_analytic(gs_ctx* ctx, int64_t n_iters, int32_t reps, int64_t* batch_out, gs_model* model_out) {
    if (!ctx || n_iters < 10 || reps < 1 || !batch_out)
        return ctx_fail(ctx, GS_ERR_INVALID_ARG, "gs_pick_analytic: need n_iters >= 10, reps >= 1 and batch_out");
    // the graph batch sizes of the paper's sweep (Sec. IV) that fit in the run
    std::vector<int64_t> S;
    for (int64_t s : {1, 10, 50, 100, 500, 1000})
        if (s <= n_iters) S.push_back(s);
    gs_model m;
    gs_status st = gs_model_calibrate(ctx, n_iters, S.data(), (int32_t)S.size(), reps, &m);
    if (st != GS_OK) return st;
    st = gs_model_pick(&m, S.data(), (int32_t)S.size(), batch_out, nullptr);
    if (st != GS_OK) return ctx_fail(ctx, st, gs_last_error(nullptr));
    if (model_out) *model_out = m;
    return GS_OK;
}

}  // extern "C"
