// Many independent 2D thermal grids of uneven sizes advanced together.
//
// GS_MULTI_FUSED: one persistent kernel per iteration covers every
// (instance, tile) work item (largest instances first); with batch_size S > 0
// the S launches are recorded into a graph by stream capture (the paper's
// Sec. II alternative to manual creation) and replayed, with a cached
// remainder graph for n mod S.
// GS_MULTI_SEPARATE: the baseline, each instance stepped by its own per-step
// (or graph-batched) launches, instance after instance on the same stream.
// Both give bit-identical results: the fused kernel runs the same tile code.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

using namespace gs;

struct gs_multi {
    std::vector<gs_ctx*> inst;
    std::vector<int64_t> nx, ny;
    gs_dtype dt;
    gs_bc bc;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    gs_heat_coeffs hc{0.5f, 0.1f, 0.1f, 0.01f, 0.05f, 80.0f};
    gs_multi_plan plan{};
    int parity = 0;
    MultiInstance* d_desc = nullptr;    // device descriptor table (depth-1 items)
    MultiInstance* d_desc_t = nullptr;  // the same for the depth-t items
    bool table_ok = false;
    LaunchDesc desc[2], desc_t[2];
    std::map<std::pair<int64_t, int>, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;
    gs_stats stats{};
    std::string err;
};

namespace {

gs_status mfail(gs_multi* m, gs_status s, const std::string& msg) {
    if (m) m->err = msg;
    return s;
}

gs_status mcuda(gs_multi* m, cudaError_t e, const char* what) {
    return mfail(m, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define GS_MCUDA(m, call)                                       \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return mcuda((m), e_, #call);    \
    } while (0)

gs_status from_ctx(gs_multi* m, gs_status st, int i) {
    if (st != GS_OK) m->err = "instance " + std::to_string(i) + ": " + gs_last_error(m->inst[i]);
    return st;
}

void drop_graphs(gs_multi* m) {
    for (auto& kv : m->graphs) {
        cudaGraphExecDestroy(kv.second.second);
        cudaGraphDestroy(kv.second.first);
    }
    m->graphs.clear();
}

void invalidate(gs_multi* m) {
    drop_graphs(m);
    m->table_ok = false;
}

int vec_elems(gs_dtype dt) { return dt == GS_F32 ? 4 : 8; }

// Build one descriptor table (largest instances first) for work items of
// kernel `variant` at temporal depth `depth`, and its two launch descriptors
// (one per buffer parity).
gs_status build_table(gs_multi* m, int variant, int depth, MultiInstance** d_table, LaunchDesc (&desc)[2]) {
    const int n = (int)m->inst.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return m->nx[a] * m->ny[a] > m->nx[b] * m->ny[b]; });
    const bool col = (variant == GS_KERNEL_COLUMN);
    const int span = heat_multi_span(m->dt, variant, depth, m->plan.block_x);
    const int item_rows = heat_multi_item_rows(m->dt, variant, depth, m->plan.rows);
    std::vector<MultiInstance> host(n);
    int item = 0;
    double step_bytes = 0.0;  // one step reads T and P and writes T of every instance
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        void* t0;
        void* t1;
        void* p;
        int64_t pt0, pt1, pp;
        ctx_field(m->inst[i], GS_FIELD_T0, &t0, &pt0);
        ctx_field(m->inst[i], GS_FIELD_T1, &t1, &pt1);
        ctx_field(m->inst[i], GS_FIELD_P, &p, &pp);
        if (!t0 || !t1 || !p)
            return mfail(m, GS_ERR_STATE, "instance " + std::to_string(i) + ": T0, T1 and P must be bound");
        if (pt0 != pt1) return mfail(m, GS_ERR_STATE, "instance " + std::to_string(i) + ": T0/T1 pitch differ");
        MultiInstance& d = host[k];
        d.T0 = t0;
        d.T1 = t1;
        d.P = p;
        d.pitch = pt0;
        d.p_pitch = pp;
        d.nx = (int)m->nx[i];
        d.ny = (int)m->ny[i];
        const int ntx = (d.nx + span - 1) / span;
        const int nty = (d.ny + item_rows - 1) / item_rows;
        d.first_item = item;
        d.n_items = ntx * nty;
        item += d.n_items;
        step_bytes += (double)ctx_elem_bytes(m->inst[i]) * ((double)pt0 * d.ny * 2 + (double)pp * d.ny);
    }
    const bool alt = traverse_alternates(m->plan.traverse, step_bytes);
    if (!*d_table) GS_MCUDA(m, gs_malloc(d_table, sizeof(MultiInstance) * n));
    GS_MCUDA(m, cudaMemcpyAsync(*d_table, host.data(), sizeof(MultiInstance) * n, cudaMemcpyHostToDevice,
                                m->stream));
    GS_MCUDA(m, cudaStreamSynchronize(m->stream));
    const void* f = heat_multi_func(m->dt, m->bc, variant, depth);
    if (!f) return mfail(m, GS_ERR_UNSUPPORTED, "no instance-batch kernel for this plan");
    const dim3 block = col ? dim3(32, m->plan.rows, 1) : dim3(m->plan.block_x, 1, 1);
    int blocks = m->plan.blocks;
    if (blocks <= 0) {
        int occ = 0;
        GS_MCUDA(m, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, (int)(block.x * block.y), 0));
        blocks = std::max(1, occ) * device_sm_count();
    }
    blocks = std::max(1, std::min(blocks, item));
    for (int par = 0; par < 2; ++par) {
        MultiArgs a{};
        a.desc = *d_table;
        a.n_inst = n;
        a.total_items = item;
        a.rows = m->plan.rows;
        a.parity = par;
        a.rev = (alt && par == 1) ? 1 : 0;
        a.c = HeatCoef{m->hc.k, m->hc.cx, m->hc.cy, m->hc.cz, m->hc.cz2, m->hc.t_amb};
        LaunchDesc& d = desc[par];
        d.func = f;
        d.grid = dim3(blocks, 1, 1);
        d.block = block;
        d.smem = 0;
        d.set_args(a);
    }
    return GS_OK;
}

// The depth-1 table and, for a temporally blocked plan, the depth-t one.
gs_status ensure_table(gs_multi* m) {
    if (m->table_ok) return GS_OK;
    gs_status st = build_table(m, m->plan.kernel, 1, &m->d_desc, m->desc);
    if (st != GS_OK) return st;
    if (m->plan.temporal_depth > 1) {
        st = build_table(m, m->plan.kernel, m->plan.temporal_depth, &m->d_desc_t, m->desc_t);
        if (st != GS_OK) return st;
    }
    m->table_ok = true;
    return GS_OK;
}

cudaError_t launch_fused(gs_multi* m, int parity, bool temporal) {
    LaunchDesc& d = temporal ? m->desc_t[parity] : m->desc[parity];
    void* args[1] = {d.arg_ptr()};
    if (!m->plan.use_pdl) return cudaLaunchKernel(d.func, d.grid, d.block, args, d.smem, m->stream);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = d.grid;
    cfg.blockDim = d.block;
    cfg.dynamicSmemBytes = d.smem;
    cfg.stream = m->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, d.func, args);
}

// The fused launches of n iterations from parity p: n / t depth-t launches,
// then n % t depth-1 launches; each flips the parity.  Returns the launches
// issued in *count and the final parity in *p_out.
cudaError_t launch_iterations(gs_multi* m, int64_t n, int p, int64_t* count, int* p_out) {
    const int t = m->plan.temporal_depth;
    const int64_t q = (t > 1) ? n / t : 0;
    const int64_t r = n - q * t;
    cudaError_t err = cudaSuccess;
    for (int64_t i = 0; i < q && err == cudaSuccess; ++i, p ^= 1) err = launch_fused(m, p, true);
    for (int64_t i = 0; i < r && err == cudaSuccess; ++i, p ^= 1) err = launch_fused(m, p, false);
    *count = q + r;
    *p_out = p;
    return err;
}

int64_t launches_for(const gs_multi* m, int64_t n) {
    const int t = m->plan.temporal_depth;
    const int64_t q = (t > 1) ? n / t : 0;
    return q + (n - q * t);
}

// Record the launches of S iterations from parity p into a graph by stream
// capture.
gs_status capture_graph(gs_multi* m, int64_t S, int p, cudaGraphExec_t* out) {
    auto key = std::make_pair(S, p);
    auto it = m->graphs.find(key);
    if (it != m->graphs.end()) {
        *out = it->second.second;
        return GS_OK;
    }
    GS_MCUDA(m, cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    int64_t count = 0;
    int p_end = p;
    cudaError_t err = launch_iterations(m, S, p, &count, &p_end);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(m->stream, &g);
    if (err != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return mcuda(m, err != cudaSuccess ? err : e2, "stream capture of the fused multi-instance launches");
    }
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiateWithFlags(&exec, g, 0);
    if (err == cudaSuccess) err = cudaGraphUpload(exec, m->stream);
    if (err != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
        return mcuda(m, err, "instantiate/upload of the captured graph");
    }
    m->graphs[key] = std::make_pair(g, exec);
    m->stats.graphs_built += 1;
    *out = exec;
    return GS_OK;
}

gs_status check_inst(gs_multi* m, int32_t i) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (i < 0 || i >= (int32_t)m->inst.size()) return mfail(m, GS_ERR_INVALID_ARG, "instance index out of range");
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_multi_create(gs_multi** out, int32_t n, const int64_t* nx, const int64_t* ny, gs_dtype storage,
                          gs_bc bc, void* stream) {
    if (out) *out = nullptr;
    if (!out || !nx || !ny || n < 1)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_create: NULL argument or n < 1");
    if (storage != GS_F32 && storage != GS_BF16 && storage != GS_F16)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_create: unknown storage dtype");
    if (bc != GS_BC_CLAMP && bc != GS_BC_DIRICHLET0)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_create: bc must be clamp or Dirichlet-0");
    int64_t items = 0;
    for (int i = 0; i < n; ++i) {
        if (nx[i] < 1 || ny[i] < 1 || nx[i] > (1 << 20) || ny[i] > (1 << 20))
            return global_fail(GS_ERR_INVALID_ARG,
                               "gs_multi_create: instance " + std::to_string(i) + ": sizes must be in [1, 2^20]");
        items += (nx[i] + 127) / 128 * ny[i];
    }
    if (items >= (int64_t(1) << 31))
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_create: more than 2^31 work items");
    gs_multi* m = new (std::nothrow) gs_multi();
    if (!m) return global_fail(GS_ERR_OOM, "gs_multi_create: host allocation failed");
    m->dt = storage;
    m->bc = bc;
    m->plan.block_x = 64;
    m->plan.rows = 8;
    m->plan.kernel = GS_KERNEL_MARCH;
    m->plan.temporal_depth = 1;
    cudaError_t e = cudaSuccess;
    if (stream) {
        m->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        m->own_stream = (e == cudaSuccess);
    }
    if (e != cudaSuccess) {
        gs_multi_destroy(m);
        return global_fail(GS_ERR_CUDA, std::string("gs_multi_create: stream creation: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < n; ++i) {
        gs_ctx* c = nullptr;
        gs_status st = gs_create(&c, GS_HEAT2D, nx[i], ny[i], 1, storage, bc, m->stream);
        if (st != GS_OK) {
            gs_multi_destroy(m);
            return st;
        }
        m->inst.push_back(c);
        m->nx.push_back(nx[i]);
        m->ny.push_back(ny[i]);
    }
    *out = m;
    return GS_OK;
}

gs_status gs_multi_destroy(gs_multi* m) {
    if (!m) return GS_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    drop_graphs(m);
    for (gs_ctx* c : m->inst) gs_destroy(c);
    if (m->d_desc) cudaFree(m->d_desc);
    if (m->d_desc_t) cudaFree(m->d_desc_t);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return GS_OK;
}

const char* gs_multi_last_error(const gs_multi* m) { return m ? m->err.c_str() : ""; }

gs_status gs_multi_set_heat_coeffs(gs_multi* m, const gs_heat_coeffs* c) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (!c) return mfail(m, GS_ERR_INVALID_ARG, "NULL argument");
    for (size_t i = 0; i < m->inst.size(); ++i) {
        gs_status st = gs_set_heat_coeffs(m->inst[i], c);
        if (st != GS_OK) return from_ctx(m, st, (int)i);
    }
    m->hc = *c;
    invalidate(m);
    return GS_OK;
}

gs_status gs_multi_set_plan(gs_multi* m, const gs_multi_plan* p) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (!p) return mfail(m, GS_ERR_INVALID_ARG, "NULL argument");
    gs_multi_plan q = *p;
    // MARCH tiles measured faster here: a persistent loop over small column
    // tiles exposes one full load round trip per work item
    if (q.kernel == GS_KERNEL_AUTO) q.kernel = GS_KERNEL_MARCH;
    if (q.kernel != GS_KERNEL_COLUMN && q.kernel != GS_KERNEL_MARCH)
        return mfail(m, GS_ERR_INVALID_ARG, "kernel must be GS_KERNEL_COLUMN or GS_KERNEL_MARCH");
    if (q.block_x == 0) q.block_x = 64;
    if (q.rows == 0) q.rows = (q.kernel == GS_KERNEL_COLUMN) ? 4 : 8;
    if (q.block_x < 32 || q.block_x > 512 || q.block_x % 32)
        return mfail(m, GS_ERR_INVALID_ARG, "block_x must be a multiple of 32 in [32, 512]");
    if (q.kernel == GS_KERNEL_COLUMN && q.rows > 8)
        return mfail(m, GS_ERR_INVALID_ARG, "COLUMN tiles take rows <= 8");
    if (q.rows < 1 || q.blocks < 0 || (q.use_pdl != 0 && q.use_pdl != 1))
        return mfail(m, GS_ERR_INVALID_ARG, "rows >= 1, blocks >= 0, use_pdl in {0, 1}");
    if (q.traverse < GS_TRAVERSE_AUTO || q.traverse > GS_TRAVERSE_ALTERNATE)
        return mfail(m, GS_ERR_INVALID_ARG, "traverse must be a gs_traverse value");
    if (q.temporal_depth == 0) q.temporal_depth = 1;
    if (q.temporal_depth != 1 && q.temporal_depth != 2 && q.temporal_depth != 4)
        return mfail(m, GS_ERR_INVALID_ARG, "temporal_depth must be 1, 2 or 4");
    if (q.temporal_depth > 1 && q.kernel != GS_KERNEL_COLUMN)
        return mfail(m, GS_ERR_INVALID_ARG, "temporal_depth > 1 runs COLUMN tiles only");
    gs_plan sp{};
    sp.block_x = q.block_x;
    sp.rows = q.rows;
    sp.temporal_depth = 1;
    sp.use_pdl = q.use_pdl;
    sp.traverse = q.traverse;
    sp.kernel = GS_KERNEL_MARCH;
    for (size_t i = 0; i < m->inst.size(); ++i) {
        gs_status st = gs_set_plan(m->inst[i], &sp);
        if (st != GS_OK) return from_ctx(m, st, (int)i);
    }
    m->plan = q;
    invalidate(m);
    return GS_OK;
}

gs_status gs_multi_bind_field(gs_multi* m, int32_t i, gs_field id, void* ptr, int64_t pitch) {
    gs_status st = check_inst(m, i);
    if (st != GS_OK) return st;
    if (id == GS_FIELD_T) return mfail(m, GS_ERR_INVALID_ARG, "bind T0/T1 explicitly");
    st = gs_bind_field(m->inst[i], id, ptr, pitch);
    if (st != GS_OK) return from_ctx(m, st, i);
    invalidate(m);
    return GS_OK;
}

gs_status gs_multi_upload(gs_multi* m, int32_t i, gs_field id, const float* host, int64_t n) {
    gs_status st = check_inst(m, i);
    if (st != GS_OK) return st;
    return from_ctx(m, gs_upload(m->inst[i], id, host, n), i);
}

gs_status gs_multi_read_field(gs_multi* m, int32_t i, gs_field id, float* host_out, int64_t n) {
    gs_status st = check_inst(m, i);
    if (st != GS_OK) return st;
    return from_ctx(m, gs_read_field(m->inst[i], id, host_out, n), i);
}

gs_status gs_multi_get_parity(const gs_multi* m, int32_t* out) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (!out) return global_fail(GS_ERR_INVALID_ARG, "NULL output pointer");
    *out = m->parity;
    return GS_OK;
}

gs_status gs_multi_step(gs_multi* m, int64_t n_iters, int64_t batch_size, gs_multi_mode mode) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (n_iters < 0 || batch_size < 0) return mfail(m, GS_ERR_INVALID_ARG, "n_iters and batch_size must be >= 0");
    if (mode != GS_MULTI_FUSED && mode != GS_MULTI_SEPARATE) return mfail(m, GS_ERR_INVALID_ARG, "unknown mode");
    if (n_iters == 0) return GS_OK;
    if (mode == GS_MULTI_SEPARATE) {
        for (size_t i = 0; i < m->inst.size(); ++i) {
            gs_status st = gs_step(m->inst[i], n_iters, batch_size);
            if (st != GS_OK) return from_ctx(m, st, (int)i);
        }
        m->parity ^= (int)(n_iters & 1);
        m->stats.iterations += n_iters;
        return GS_OK;
    }
    gs_status st = ensure_table(m);
    if (st != GS_OK) return st;
    if (batch_size == 0) {
        int64_t count = 0;
        int p_end = m->parity;
        GS_MCUDA(m, launch_iterations(m, n_iters, m->parity, &count, &p_end));
        m->parity = p_end;
        m->stats.kernel_launches += count;
    } else {
        const int64_t nb = n_iters / batch_size, r = n_iters % batch_size;
        for (int64_t b = 0; b < nb; ++b) {
            cudaGraphExec_t ex;
            st = capture_graph(m, batch_size, m->parity, &ex);
            if (st != GS_OK) return st;
            GS_MCUDA(m, cudaGraphLaunch(ex, m->stream));
            m->stats.graph_launches += 1;
            m->parity ^= (int)(launches_for(m, batch_size) & 1);
        }
        if (r) {
            cudaGraphExec_t ex;
            st = capture_graph(m, r, m->parity, &ex);
            if (st != GS_OK) return st;
            GS_MCUDA(m, cudaGraphLaunch(ex, m->stream));
            m->stats.graph_launches += 1;
            m->parity ^= (int)(launches_for(m, r) & 1);
        }
    }
    // keep each instance context's view of the current buffer in step
    for (gs_ctx* c : m->inst) gs_set_parity(c, m->parity);
    m->stats.iterations += n_iters;
    return GS_OK;
}

gs_status gs_multi_get_plan(const gs_multi* m, gs_multi_plan* out) {
    if (!m || !out) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch or output pointer");
    *out = m->plan;
    return GS_OK;
}

gs_status gs_multi_candidates(const gs_multi* m, gs_multi_tune_candidate* out, int32_t capacity, int32_t* n_out) {
    if (!m || !n_out || capacity < 0 || (capacity > 0 && !out))
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_candidates: NULL argument or negative capacity");
    // (kernel, block_x, rows, depth) of each plan
    static const int plans[][4] = {
        {GS_KERNEL_MARCH, 64, 4, 1},  {GS_KERNEL_MARCH, 64, 8, 1},  {GS_KERNEL_MARCH, 64, 16, 1},
        {GS_KERNEL_MARCH, 128, 4, 1}, {GS_KERNEL_MARCH, 128, 8, 1}, {GS_KERNEL_MARCH, 128, 16, 1},
        {GS_KERNEL_COLUMN, 64, 2, 1}, {GS_KERNEL_COLUMN, 64, 4, 1}, {GS_KERNEL_COLUMN, 64, 8, 1},
        {GS_KERNEL_COLUMN, 64, 1, 2}, {GS_KERNEL_COLUMN, 64, 2, 2}, {GS_KERNEL_COLUMN, 64, 4, 2},
        {GS_KERNEL_COLUMN, 64, 1, 4}, {GS_KERNEL_COLUMN, 64, 2, 4}};
    static const int64_t batches[] = {0, 10, 100, 1000};
    const int32_t n = (int32_t)(sizeof(plans) / sizeof(plans[0]) * (sizeof(batches) / sizeof(batches[0])));
    *n_out = n;
    if (!out) return GS_OK;
    if (capacity < n)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_candidates: capacity below the " + std::to_string(n) +
                                                   " candidates");
    int32_t i = 0;
    for (const auto& pl : plans)
        for (int64_t S : batches) {
            gs_multi_tune_candidate& c = out[i++];
            c = gs_multi_tune_candidate{};
            c.plan.kernel = pl[0];
            c.plan.block_x = pl[1];
            c.plan.rows = pl[2];
            c.plan.temporal_depth = pl[3];
            c.batch_size = S;
        }
    return GS_OK;
}

namespace {

// Capture every graph gs_multi_step(n, S, FUSED) uses from the current
// parity: the batch graph (both parities when a batch flips it and more
// than one batch runs) and the remainder graph.
gs_status capture_for_run(gs_multi* m, int64_t n, int64_t S) {
    gs_status st = ensure_table(m);
    if (st != GS_OK) return st;
    const int p = m->parity;
    const int64_t nb = n / S, r = n % S;
    const int fl = (int)(launches_for(m, S) & 1);
    cudaGraphExec_t ex;
    if (nb > 0) {
        st = capture_graph(m, S, p, &ex);
        if (st == GS_OK && fl && nb > 1) st = capture_graph(m, S, p ^ 1, &ex);
        if (st != GS_OK) return st;
    }
    if (r > 0) return capture_graph(m, r, p ^ (fl & (int)(nb & 1)), &ex);
    return GS_OK;
}

}  // namespace

gs_status gs_multi_autotune(gs_multi* m, int64_t n_iters, int32_t reps, const gs_multi_tune_candidate* cands,
                            int32_t n_cands, gs_multi_tune_result* results, int32_t* best_index) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (!cands || !results || n_cands < 1 || n_iters < 1 || reps < 1)
        return mfail(m, GS_ERR_INVALID_ARG, "gs_multi_autotune: NULL pointer, or n_cands/n_iters/reps < 1");
    // snapshot every instance's current buffer
    const int n = (int)m->inst.size();
    std::vector<void*> snap(n, nullptr), cur(n, nullptr);
    std::vector<size_t> bytes(n, 0);
    gs_status fatal = GS_OK;
    for (int i = 0; i < n && fatal == GS_OK; ++i) {
        int64_t pitch;
        ctx_field(m->inst[i], m->parity ? GS_FIELD_T1 : GS_FIELD_T0, &cur[i], &pitch);
        void* pp;
        int64_t ppitch;
        ctx_field(m->inst[i], GS_FIELD_P, &pp, &ppitch);
        void* other;
        int64_t opitch;
        ctx_field(m->inst[i], m->parity ? GS_FIELD_T0 : GS_FIELD_T1, &other, &opitch);
        if (!cur[i] || !pp || !other) {
            fatal = mfail(m, GS_ERR_STATE, "gs_multi_autotune: instance " + std::to_string(i) + ": unbound field");
            break;
        }
        bytes[i] = (size_t)pitch * (size_t)m->ny[i] * ctx_elem_bytes(m->inst[i]);
        cudaError_t e = gs_malloc(&snap[i], bytes[i]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(snap[i], cur[i], bytes[i], cudaMemcpyDeviceToDevice, m->stream);
        if (e != cudaSuccess) fatal = mcuda(m, e, "gs_multi_autotune snapshot");
    }
    if (fatal == GS_OK) {
        cudaError_t e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) fatal = mcuda(m, e, "gs_multi_autotune snapshot");
    }
    if (fatal != GS_OK) {
        for (void* b : snap)
            if (b) cudaFree(b);
        return fatal;
    }
    const gs_multi_plan saved = m->plan;
    const int saved_parity = m->parity;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    double best_total = INFINITY;
    int32_t best = -1;
    for (int32_t c = 0; c < n_cands && fatal == GS_OK; ++c) {
        gs_multi_tune_result& r = results[c];
        r = gs_multi_tune_result{};
        r.plan = cands[c].plan;
        r.batch_size = cands[c].batch_size;
        r.exec_ms_per_iter = INFINITY;
        r.total_ms = INFINITY;
        const int64_t S = cands[c].batch_size;
        gs_status rs = (S < 0) ? GS_ERR_INVALID_ARG : gs_multi_set_plan(m, &cands[c].plan);
        r.status = rs;
        if (rs != GS_OK) continue;  // not runnable: skipped
        r.plan = m->plan;
        if (S > 0) {
            cudaError_t e = cudaStreamSynchronize(m->stream);
            const auto t0 = std::chrono::steady_clock::now();
            rs = (e == cudaSuccess) ? capture_for_run(m, n_iters, S) : mcuda(m, e, "gs_multi_autotune");
            if (rs == GS_OK) {
                e = cudaStreamSynchronize(m->stream);
                if (e != cudaSuccess) rs = mcuda(m, e, "gs_multi_autotune build");
            }
            r.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
        // warm-up run, then timed runs
        if (rs == GS_OK) rs = gs_multi_step(m, n_iters, S, GS_MULTI_FUSED);
        if (rs == GS_OK) rs = gs_multi_sync(m);
        double best_ms = INFINITY;
        for (int32_t k = 0; k < reps && rs == GS_OK; ++k) {
            cudaEventRecord(ev0, m->stream);
            rs = gs_multi_step(m, n_iters, S, GS_MULTI_FUSED);
            cudaEventRecord(ev1, m->stream);
            if (rs != GS_OK) break;
            cudaError_t e = cudaEventSynchronize(ev1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (e != cudaSuccess) {
                rs = mcuda(m, e, "gs_multi_autotune timing");
                break;
            }
            best_ms = std::min(best_ms, (double)ms);
        }
        r.status = rs;
        if (rs != GS_OK) {
            if (rs == GS_ERR_CUDA || rs == GS_ERR_OOM) fatal = rs;
            continue;
        }
        r.exec_ms_per_iter = best_ms / (double)n_iters;
        r.total_ms = r.build_seconds * 1e3 + best_ms;
        if (r.total_ms < best_total) {
            best_total = r.total_ms;
            best = c;
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    // restore the plan, the parity and every instance's state
    const std::string fatal_msg = m->err;
    gs_multi_set_plan(m, &saved);
    cudaError_t e = cudaStreamSynchronize(m->stream);
    m->parity = saved_parity;
    for (gs_ctx* c : m->inst) gs_set_parity(c, saved_parity);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(cur[i], snap[i], bytes[i], cudaMemcpyDeviceToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    for (void* b : snap) cudaFree(b);
    if (fatal != GS_OK) return mfail(m, fatal, fatal_msg);
    if (e != cudaSuccess) return mcuda(m, e, "gs_multi_autotune restore");
    if (best_index) *best_index = best;
    if (best < 0) return mfail(m, GS_ERR_UNSUPPORTED, "gs_multi_autotune: no candidate could run");
    return GS_OK;
}

gs_status gs_multi_sync(gs_multi* m) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    GS_MCUDA(m, cudaStreamSynchronize(m->stream));
    return GS_OK;
}

gs_status gs_multi_get_stats(const gs_multi* m, gs_stats* out) {
    if (!m) return global_fail(GS_ERR_INVALID_ARG, "NULL instance batch");
    if (!out) return global_fail(GS_ERR_INVALID_ARG, "NULL output pointer");
    *out = m->stats;
    for (gs_ctx* c : m->inst) {
        gs_stats s;
        gs_get_stats(c, &s);
        out->kernel_launches += s.kernel_launches;
        out->graph_launches += s.graph_launches;
        out->graphs_built += s.graphs_built;
    }
    return GS_OK;
}

}  // extern "C"
