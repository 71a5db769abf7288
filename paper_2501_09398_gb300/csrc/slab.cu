// Slab decomposition: one grid split along its slowest axis into sub-domains
// (slabs) with halo rows/planes, each slab a context of its own, the halos
// refreshed from the neighbours' owned rows after every launch.  This is the
// layout a grid spread over several GPUs takes (one slab per GPU, the halo
// copies peer copies); here every slab lives on the current device.
//
// Batch graphs (the paper's iteration batches, Sec. III-A, widened to a
// DAG): per launch j, one kernel node per slab, then one copy node per halo
// (a 2D copy: 1 chunk for a thermal field, the 3 components of an FDTD field
// at their common stride).  A slab's kernel j+1 depends on its kernel j and
// on every copy of exchange j that writes or reads its fields; a copy
// depends on the kernels j of both slabs it joins.  So neighbouring slabs
// synchronise only through their halos, and the slabs' kernels of one step
// may run at once.
//
// Why the result is bit-identical to the undivided grid: every owned cell is
// updated by the same kernel code from the same neighbour values.  A slab
// computes its halo rows too, with the slab edge taken as a boundary, so
// they go wrong; a depth-t launch spreads that error t rows inward, which
// the t-row halo absorbs, and the exchange overwrites the halos with the
// neighbours' owned rows before the next launch reads them.  FDTD (halo 1):
// the H update of the top owned plane reads E on the plane above (the top
// halo, refreshed after each E update); the E update of the bottom owned
// plane reads H on the plane below (the bottom halo, refreshed after each H
// update); the slab's own k walls lie on halo planes, which owned updates
// never read.
#include <algorithm>
#include <chrono>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

using namespace gs;

namespace {

struct SlabGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
};

// One halo copy after a launch: `height` chunks of `width` bytes, `stride`
// bytes apart in both slabs (1 chunk for thermal fields, the 3 components
// of an FDTD field).
struct HaloCopy {
    int src, dst;  // slab indices
    char* from;
    char* to;
    size_t width, height, stride;
};

}  // namespace

struct gs_slab {
    gs_kind kind;
    int64_t nx, ny, nz;
    gs_dtype dt;
    gs_bc bc;
    int K = 1;
    int halo = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<gs_ctx*> ctx;
    std::vector<int64_t> first, count;  // owned units (rows 2D, planes 3D / FDTD arrays), global
    std::vector<int64_t> lo, n_local;   // global index of local unit 0; local units held
    std::vector<char*> mem;             // one allocation per slab
    int64_t pitch = 0;                  // elements per row
    size_t unit_bytes = 0;              // bytes per row (2D) / plane (3D, FDTD)
    size_t tbytes = 0;                  // thermal: bytes reserved per T buffer; FDTD: per component
    int parity = 0;
    int64_t time = 0;
    gs_plan plan{};
    std::map<std::pair<int64_t, int>, SlabGraph> graphs;
    int64_t rem_S = 0;
    gs_stats stats{};
    std::string err;
};

namespace {

gs_status sfail(gs_slab* s, gs_status st, const std::string& msg) {
    if (s) s->err = msg;
    else global_fail(st, msg);
    return st;
}

gs_status scuda(gs_slab* s, cudaError_t e, const char* what) {
    return sfail(s, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define GS_SCUDA(s, call)                                     \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return scuda((s), e_, #call);  \
    } while (0)

gs_status from_slab(gs_slab* s, gs_status st, int k) {
    if (st != GS_OK) s->err = "slab " + std::to_string(k) + ": " + gs_last_error(s->ctx[k]);
    return st;
}

bool is_fdtd(const gs_slab* s) { return s->kind == GS_FDTD3D; }
size_t elem_bytes(gs_dtype dt) { return dt == GS_F32 ? 4 : 2; }
size_t round256(size_t b) { return (b + 255) / 256 * 256; }

void drop_graphs(gs_slab* s) {
    for (auto& kv : s->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    s->graphs.clear();
    s->rem_S = 0;
}

// Base address of thermal buffer b (0, 1: T0, T1; 2: P) or FDTD component c.
char* field_base(const gs_slab* s, int k, int which) { return s->mem[k] + (size_t)which * s->tbytes; }

// The halo copies after launch j of a sequence that started at parity p0.
void copies_after(const gs_slab* s, int64_t j, int p0, std::vector<HaloCopy>* out) {
    out->clear();
    const int K = s->K;
    if (K < 2) return;
    if (!is_fdtd(s)) {
        const int b = (int)((p0 + j + 1) & 1);  // buffer the launch wrote
        const size_t w = (size_t)s->halo * s->unit_bytes;
        for (int k = 1; k < K; ++k) {  // bottom halo of k <- top owned rows of k-1
            const int64_t src_unit = s->first[k] - s->halo - s->lo[k - 1];
            out->push_back(HaloCopy{k - 1, k, field_base(s, k - 1, b) + src_unit * s->unit_bytes, field_base(s, k, b),
                                    w, 1, w});
        }
        for (int k = 0; k + 1 < K; ++k) {  // top halo of k <- bottom owned rows of k+1
            const int64_t dst_unit = s->first[k] + s->count[k] - s->lo[k];
            const int64_t src_unit = s->first[k + 1] - s->lo[k + 1];
            out->push_back(HaloCopy{k + 1, k, field_base(s, k + 1, b) + src_unit * s->unit_bytes,
                                    field_base(s, k, b) + dst_unit * s->unit_bytes, w, 1, w});
        }
        return;
    }
    const size_t w = s->unit_bytes;
    if ((j & 1) == 0) {
        // after H: the plane below each slab (its local plane 0) <- the lower
        // neighbour's last owned plane, components Hx, Hy, Hz
        for (int k = 1; k < K; ++k) {
            const int64_t src_unit = s->first[k] - 1 - s->lo[k - 1];
            out->push_back(HaloCopy{k - 1, k, field_base(s, k - 1, 3) + src_unit * w, field_base(s, k, 3), w, 3,
                                    s->tbytes});
        }
    } else {
        // after E: the plane above each slab <- the upper neighbour's first
        // owned plane, components Ex, Ey, Ez
        for (int k = 0; k + 1 < K; ++k) {
            const int64_t dst_unit = s->first[k] + s->count[k] - s->lo[k];
            const int64_t src_unit = s->first[k + 1] - s->lo[k + 1];
            out->push_back(HaloCopy{k + 1, k, field_base(s, k + 1, 0) + src_unit * w, field_base(s, k, 0) + dst_unit * w,
                                    w, 3, s->tbytes});
        }
    }
}

cudaMemcpy3DParms copy_params(const HaloCopy& c) {
    cudaMemcpy3DParms p{};
    p.srcPtr = make_cudaPitchedPtr(c.from, c.stride, c.width, c.height);
    p.dstPtr = make_cudaPitchedPtr(c.to, c.stride, c.width, c.height);
    p.extent = make_cudaExtent(c.width, c.height, 1);
    p.kind = cudaMemcpyDeviceToDevice;
    return p;
}

gs_status prepare(gs_slab* s) {
    for (int k = 0; k < s->K; ++k) {
        gs_status st = ctx_prepare(s->ctx[k]);
        if (st != GS_OK) return from_slab(s, st, k);
    }
    return GS_OK;
}

// Every slab's launch sequence of n iterations from parity p (equal lengths).
void launch_lists(gs_slab* s, int64_t n, int p, std::vector<std::vector<LaunchDesc*>>* lists) {
    lists->assign(s->K, {});
    for (int k = 0; k < s->K; ++k) ctx_launch_list(s->ctx[k], n, p, &(*lists)[k]);
}

// Build the batch graph of S iterations from parity p.
gs_status build_graph(gs_slab* s, int64_t S, int p, SlabGraph* out) {
    std::vector<std::vector<LaunchDesc*>> lists;
    launch_lists(s, S, p, &lists);
    const size_t L = lists[0].size();
    cudaGraph_t g = nullptr;
    GS_SCUDA(s, cudaGraphCreate(&g, 0));
    cudaError_t err = cudaSuccess;
    std::vector<cudaGraphNode_t> prev_k(s->K, nullptr);
    std::vector<std::vector<cudaGraphNode_t>> prev_c(s->K), next_c(s->K);
    std::vector<cudaGraphNode_t> cur_k(s->K, nullptr);
    std::vector<HaloCopy> copies;
    int64_t nodes = 0;
    for (size_t j = 0; j < L && err == cudaSuccess; ++j) {
        for (int k = 0; k < s->K && err == cudaSuccess; ++k) {
            LaunchDesc& d = *lists[k][j];
            std::vector<cudaGraphNode_t> deps(prev_c[k]);
            if (prev_k[k]) deps.push_back(prev_k[k]);
            cudaKernelNodeParams np{};
            void* args[1] = {d.arg_ptr()};
            np.func = const_cast<void*>(d.func);
            np.gridDim = d.grid;
            np.blockDim = d.block;
            np.sharedMemBytes = (unsigned)d.smem;
            np.kernelParams = args;
            err = gs_graph_add_kernel_node(&cur_k[k], g, deps.empty() ? nullptr : deps.data(), deps.size(), &np);
            ++nodes;
        }
        copies_after(s, (int64_t)j, p, &copies);
        for (auto& v : next_c) v.clear();
        for (const HaloCopy& c : copies) {
            if (err != cudaSuccess) break;
            cudaGraphNode_t deps[2] = {cur_k[c.src], cur_k[c.dst]};
            const cudaMemcpy3DParms cp = copy_params(c);
            cudaGraphNode_t node;
            err = cudaGraphAddMemcpyNode(&node, g, deps, 2, &cp);
            next_c[c.src].push_back(node);
            next_c[c.dst].push_back(node);
            ++nodes;
        }
        prev_k = cur_k;
        prev_c.swap(next_c);
    }
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        return scuda(s, err, "slab batch graph construction");
    }
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiateWithFlags(&exec, g, 0);
    if (err == cudaSuccess) err = cudaGraphUpload(exec, s->stream);
    if (err != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
        return scuda(s, err, "slab batch graph instantiate/upload");
    }
    out->graph = g;
    out->exec = exec;
    out->nodes = nodes;
    s->stats.graphs_built += 1;
    return GS_OK;
}

gs_status ensure_graph(gs_slab* s, int64_t S, int p) {
    auto key = std::make_pair(S, p);
    if (s->graphs.count(key)) return GS_OK;
    SlabGraph e;
    gs_status st = build_graph(s, S, p, &e);
    if (st != GS_OK) return st;
    s->graphs.emplace(key, e);
    return GS_OK;
}

// Every graph gs_slab_step(n, S) launches, built before the first launch
// (a failed build leaves the set as it was).
gs_status prepare_graphs(gs_slab* s, int64_t n, int64_t S) {
    const int64_t nb = n / S, r = n % S;
    const int fl = ctx_flip(s->ctx[0], S);
    int p = s->parity;
    gs_status st = GS_OK;
    if (nb > 0) {
        st = ensure_graph(s, S, p);
        if (st == GS_OK && fl && nb > 1) st = ensure_graph(s, S, p ^ 1);
        if (st != GS_OK) return st;
        p ^= fl & (int)(nb & 1);
    }
    if (r > 0) st = ensure_graph(s, r, p);
    return st;
}

gs_status launch_graphs(gs_slab* s, int64_t S, int64_t count) {
    const int fl = ctx_flip(s->ctx[0], S);
    for (int64_t i = 0; i < count; ++i) {
        gs_status st = ensure_graph(s, S, s->parity);
        if (st != GS_OK) return st;
        auto it = s->graphs.find(std::make_pair(S, s->parity));
        GS_SCUDA(s, cudaGraphLaunch(it->second.exec, s->stream));
        s->stats.graph_launches += 1;
        s->stats.last_build_nodes = it->second.nodes;
        s->parity ^= fl;
    }
    return GS_OK;
}

// Per-step launches: every slab's launch j, then the halo copies.
gs_status run_per_step(gs_slab* s, int64_t n) {
    std::vector<std::vector<LaunchDesc*>> lists;
    launch_lists(s, n, s->parity, &lists);
    std::vector<HaloCopy> copies;
    const size_t L = lists[0].size();
    for (size_t j = 0; j < L; ++j) {
        for (int k = 0; k < s->K; ++k) {
            cudaError_t e = ctx_launch(s->ctx[k], *lists[k][j]);
            if (e != cudaSuccess) return scuda(s, e, "slab kernel launch");
            s->stats.kernel_launches += 1;
        }
        copies_after(s, (int64_t)j, s->parity, &copies);
        for (const HaloCopy& c : copies)
            GS_SCUDA(s, cudaMemcpy2DAsync(c.to, c.stride, c.from, c.stride, c.width, c.height,
                                          cudaMemcpyDeviceToDevice, s->stream));
    }
    s->parity ^= ctx_flip(s->ctx[0], n);
    return GS_OK;
}

// Dense elements of one unit (row or plane) and units of the global field.
void global_units(const gs_slab* s, int field, int64_t* unit_elems, int64_t* units) {
    if (is_fdtd(s)) {
        *unit_elems = (s->nx + 1) * (s->nx + 1);
        *units = s->nz + 1;
    } else if (s->kind == GS_HEAT2D) {
        *unit_elems = s->nx;
        *units = s->ny;
    } else {
        *unit_elems = s->nx * s->ny;
        *units = (field == GS_FIELD_P) ? 1 : s->nz;
    }
}

gs_status check_field(gs_slab* s, gs_field id, int* f) {
    int v = id;
    if (!is_fdtd(s)) {
        if (v == GS_FIELD_T) v = s->parity ? GS_FIELD_T1 : GS_FIELD_T0;
        if (v != GS_FIELD_T0 && v != GS_FIELD_T1 && v != GS_FIELD_P)
            return sfail(s, GS_ERR_INVALID_ARG, "thermal slab sets hold T0, T1 (or T) and P");
    } else if (v < GS_FIELD_EX || v > GS_FIELD_HZ) {
        return sfail(s, GS_ERR_INVALID_ARG, "FDTD slab sets hold the six components");
    }
    *f = v;
    return GS_OK;
}

// A 3D slab set's power map is one plane that every slab holds whole.
bool whole_plane(const gs_slab* s, int f) { return s->kind == GS_HEAT3D && f == GS_FIELD_P; }

}  // namespace

extern "C" {

gs_status gs_slab_create(gs_slab** out, gs_kind kind, int64_t nx, int64_t ny, int64_t nz, gs_dtype storage, gs_bc bc,
                         int32_t n_slabs, int32_t halo, void* stream) {
    if (!out) return global_fail(GS_ERR_INVALID_ARG, "gs_slab_create: out is NULL");
    *out = nullptr;
    if (kind != GS_HEAT2D && kind != GS_HEAT3D && kind != GS_FDTD3D)
        return global_fail(GS_ERR_INVALID_ARG, "gs_slab_create: kind must be GS_HEAT2D, GS_HEAT3D or GS_FDTD3D");
    if (n_slabs < 1 || n_slabs > 64) return global_fail(GS_ERR_INVALID_ARG, "gs_slab_create: n_slabs must be in [1, 64]");
    if (kind == GS_FDTD3D ? halo != 1 : (halo < 1 || halo > 4))
        return global_fail(GS_ERR_INVALID_ARG, "gs_slab_create: halo must be 1 (FDTD) or in [1, 4] (thermal)");
    // the undivided grid must be a valid context (checked without a device)
    {
        gs_workload w{kind, storage, nx, ny, nz, 1};
        gs_plan p{};
        gs_status st = gs_plan_check(&w, &p, nullptr);
        if (st != GS_OK) return global_fail(st, std::string("gs_slab_create: ") + gs_last_error(nullptr));
        if (kind == GS_FDTD3D ? bc != GS_BC_PEC : (bc != GS_BC_CLAMP && bc != GS_BC_DIRICHLET0))
            return global_fail(GS_ERR_INVALID_ARG, "gs_slab_create: bc does not match the kind");
    }
    const int64_t units = (kind == GS_HEAT2D) ? ny : (kind == GS_HEAT3D ? nz : nx + 1);
    const int64_t min_own = (kind == GS_FDTD3D) ? 1 : halo;
    if (units / n_slabs < min_own)
        return global_fail(GS_ERR_INVALID_ARG, "gs_slab_create: " + std::to_string(units) + " rows/planes cannot give " +
                                                   std::to_string(n_slabs) + " slabs of at least " +
                                                   std::to_string(min_own) + " each");
    gs_slab* s = new (std::nothrow) gs_slab();
    if (!s) return global_fail(GS_ERR_OOM, "gs_slab_create: host allocation failed");
    s->kind = kind;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->dt = storage;
    s->bc = bc;
    s->K = n_slabs;
    s->halo = halo;
    const int64_t base = units / n_slabs, extra = units % n_slabs;
    int64_t at = 0;
    for (int k = 0; k < n_slabs; ++k) {
        const int64_t c = base + (k < extra ? 1 : 0);
        const int64_t hb = (k > 0) ? halo : 0, ht = (k + 1 < n_slabs) ? halo : 0;
        s->first.push_back(at);
        s->count.push_back(c);
        s->lo.push_back(at - hb);
        s->n_local.push_back(c + hb + ht);
        at += c;
    }
    cudaError_t e = cudaSuccess;
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = (e == cudaSuccess);
    }
    if (e != cudaSuccess) {
        gs_slab_destroy(s);
        return global_fail(GS_ERR_CUDA, std::string("gs_slab_create: stream: ") + cudaGetErrorString(e));
    }
    const size_t eb = elem_bytes(storage);
    gs_required_pitch(storage, kind == GS_FDTD3D ? nx + 1 : nx, &s->pitch);
    s->unit_bytes = (size_t)s->pitch * eb * (kind == GS_HEAT2D ? 1 : (kind == GS_HEAT3D ? ny : nx + 1));
    for (int k = 0; k < n_slabs; ++k) {
        gs_ctx* c = nullptr;
        gs_status st;
        if (kind == GS_HEAT2D) st = gs_create(&c, kind, nx, s->n_local[k], 1, storage, bc, s->stream);
        else if (kind == GS_HEAT3D) st = gs_create(&c, kind, nx, ny, s->n_local[k], storage, bc, s->stream);
        else st = ctx_create(&c, kind, nx, nx, s->n_local[k] - 1, storage, bc, s->stream, true);
        if (st != GS_OK) {
            const std::string why = gs_last_error(nullptr);
            gs_slab_destroy(s);
            return global_fail(st, "gs_slab_create: slab " + std::to_string(k) + ": " + why);
        }
        s->ctx.push_back(c);
    }
    // memory: per slab T0 | T1 | P (thermal) or the six components
    size_t per = 0;
    for (int k = 0; k < n_slabs; ++k)
        s->tbytes = std::max(s->tbytes, round256((size_t)s->n_local[k] * s->unit_bytes));
    if (kind == GS_FDTD3D) {
        per = 6 * s->tbytes;
    } else {
        const int64_t p_rows = (kind == GS_HEAT2D) ? *std::max_element(s->n_local.begin(), s->n_local.end()) : ny;
        const size_t pb = round256((size_t)s->pitch * eb * (size_t)p_rows);
        per = 2 * s->tbytes + pb;
    }
    for (int k = 0; k < n_slabs; ++k) {
        void* p = nullptr;
        e = gs_malloc(&p, per);
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, per, s->stream);
        if (e != cudaSuccess) {
            if (p) cudaFree(p);
            gs_slab_destroy(s);
            return global_fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                               std::string("gs_slab_create: slab memory: ") + cudaGetErrorString(e));
        }
        s->mem.push_back(static_cast<char*>(p));
        gs_status st = GS_OK;
        if (kind == GS_FDTD3D) {
            for (int f = 0; f < 6 && st == GS_OK; ++f)
                st = gs_bind_field(s->ctx[k], (gs_field)(GS_FIELD_EX + f), field_base(s, k, f), s->pitch);
            if (st == GS_OK) {
                gs_fdtd_params fp{0.5f, 0, 0, 0, 0, 1.0f, 60.0f, 20.0f};
                st = gs_set_fdtd_params(s->ctx[k], &fp);
            }
        } else {
            st = gs_bind_field(s->ctx[k], GS_FIELD_T0, field_base(s, k, 0), s->pitch);
            if (st == GS_OK) st = gs_bind_field(s->ctx[k], GS_FIELD_T1, field_base(s, k, 1), s->pitch);
            if (st == GS_OK) st = gs_bind_field(s->ctx[k], GS_FIELD_P, field_base(s, k, 2), s->pitch);
        }
        if (st != GS_OK) {
            const std::string why = gs_last_error(s->ctx[k]);
            gs_slab_destroy(s);
            return global_fail(st, "gs_slab_create: slab " + std::to_string(k) + ": " + why);
        }
    }
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        gs_slab_destroy(s);
        return global_fail(GS_ERR_CUDA, std::string("gs_slab_create: ") + cudaGetErrorString(e));
    }
    gs_get_plan(s->ctx[0], &s->plan);
    *out = s;
    return GS_OK;
}

gs_status gs_slab_destroy(gs_slab* s) {
    if (!s) return GS_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graphs(s);
    for (gs_ctx* c : s->ctx) gs_destroy(c);
    for (char* p : s->mem) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return GS_OK;
}

const char* gs_slab_last_error(const gs_slab* s) { return s ? s->err.c_str() : ""; }

gs_status gs_slab_extent(const gs_slab* s, int32_t k, int64_t* first, int64_t* count) {
    if (!s || !first || !count) return global_fail(GS_ERR_INVALID_ARG, "gs_slab_extent: NULL argument");
    if (k < 0 || k >= s->K) return global_fail(GS_ERR_INVALID_ARG, "gs_slab_extent: slab index out of range");
    *first = s->first[k];
    *count = s->count[k];
    return GS_OK;
}

gs_status gs_slab_set_heat_coeffs(gs_slab* s, const gs_heat_coeffs* c) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    for (int k = 0; k < s->K; ++k) {
        gs_status st = gs_set_heat_coeffs(s->ctx[k], c);
        if (st != GS_OK) return from_slab(s, st, k);
    }
    drop_graphs(s);
    return GS_OK;
}

gs_status gs_slab_set_fdtd_params(gs_slab* s, const gs_fdtd_params* p) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    if (!p) return sfail(s, GS_ERR_INVALID_ARG, "NULL argument");
    if (!is_fdtd(s)) return sfail(s, GS_ERR_INVALID_ARG, "not an FDTD slab set");
    if (p->src_k < 0 || p->src_k > s->nz)
        return sfail(s, GS_ERR_INVALID_ARG, "source cell outside the (N+1)^3 arrays");
    for (int k = 0; k < s->K; ++k) {
        gs_fdtd_params q = *p;
        const bool owner = p->src_k >= s->first[k] && p->src_k < s->first[k] + s->count[k];
        if (owner) {
            q.src_k = p->src_k - s->lo[k];
        } else {
            // no source here; the thread of cell (0, 0, 0) keeps the step counter
            q.src_on = 0;
            q.src_i = q.src_j = q.src_k = 0;
        }
        gs_status st = gs_set_fdtd_params(s->ctx[k], &q);
        if (st != GS_OK) return from_slab(s, st, k);
    }
    drop_graphs(s);
    return GS_OK;
}

gs_status gs_slab_set_plan(gs_slab* s, const gs_plan* plan) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    if (!plan) return sfail(s, GS_ERR_INVALID_ARG, "NULL argument");
    if (plan->graph_loop || plan->device_launch)
        return sfail(s, GS_ERR_UNSUPPORTED, "slab sets provide neither plan.graph_loop nor plan.device_launch");
    if (plan->kernel == GS_KERNEL_FUSED)
        return sfail(s, GS_ERR_UNSUPPORTED, "slab sets run the FDTD half-steps as two launches (no GS_KERNEL_FUSED)");
    if (plan->temporal_depth > s->halo)
        return sfail(s, GS_ERR_UNSUPPORTED, "plan.temporal_depth " + std::to_string(plan->temporal_depth) +
                                                " exceeds the halo of " + std::to_string(s->halo));
    gs_plan old = s->plan;
    for (int k = 0; k < s->K; ++k) {
        gs_status st = gs_set_plan(s->ctx[k], plan);
        if (st != GS_OK) {
            from_slab(s, st, k);
            for (int q = 0; q < k; ++q) gs_set_plan(s->ctx[q], &old);
            return st;
        }
    }
    gs_get_plan(s->ctx[0], &s->plan);
    drop_graphs(s);
    return GS_OK;
}

gs_status gs_slab_upload(gs_slab* s, gs_field id, const float* host, int64_t n) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    if (!host) return sfail(s, GS_ERR_INVALID_ARG, "NULL argument");
    int f;
    gs_status st = check_field(s, id, &f);
    if (st != GS_OK) return st;
    int64_t ue, units;
    global_units(s, f, &ue, &units);
    if (n != ue * units) return sfail(s, GS_ERR_INVALID_ARG, "n must equal the whole grid's dense element count " +
                                                             std::to_string(ue * units));
    for (int k = 0; k < s->K; ++k) {
        const int64_t off = whole_plane(s, f) ? 0 : s->lo[k] * ue;
        const int64_t cnt = whole_plane(s, f) ? ue : s->n_local[k] * ue;
        st = gs_upload(s->ctx[k], (gs_field)f, host + off, cnt);
        if (st != GS_OK) return from_slab(s, st, k);
    }
    return GS_OK;
}

gs_status gs_slab_read_field(gs_slab* s, gs_field id, float* host_out, int64_t n) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    if (!host_out) return sfail(s, GS_ERR_INVALID_ARG, "NULL argument");
    int f;
    gs_status st = check_field(s, id, &f);
    if (st != GS_OK) return st;
    int64_t ue, units;
    global_units(s, f, &ue, &units);
    if (n != ue * units) return sfail(s, GS_ERR_INVALID_ARG, "n must equal the whole grid's dense element count " +
                                                             std::to_string(ue * units));
    std::vector<float> tmp;
    for (int k = 0; k < s->K; ++k) {
        if (whole_plane(s, f)) {
            if (k > 0) break;
            return from_slab(s, gs_read_field(s->ctx[0], (gs_field)f, host_out, ue), 0);
        }
        tmp.resize((size_t)(s->n_local[k] * ue));
        st = gs_read_field(s->ctx[k], (gs_field)f, tmp.data(), (int64_t)tmp.size());
        if (st != GS_OK) return from_slab(s, st, k);
        std::copy(tmp.begin() + (s->first[k] - s->lo[k]) * ue, tmp.begin() + (s->first[k] - s->lo[k] + s->count[k]) * ue,
                  host_out + s->first[k] * ue);
    }
    return GS_OK;
}

gs_status gs_slab_step(gs_slab* s, int64_t n_iters, int64_t batch_size) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    if (n_iters < 0 || batch_size < 0) return sfail(s, GS_ERR_INVALID_ARG, "n_iters and batch_size must be >= 0");
    gs_status st = prepare(s);
    if (st != GS_OK) return st;
    if (n_iters == 0) return GS_OK;
    if (batch_size == 0) {
        st = run_per_step(s, n_iters);
        if (st != GS_OK) return st;
    } else {
        const int64_t nb = n_iters / batch_size, r = n_iters % batch_size;
        if (r > 0 && s->rem_S != r && s->rem_S != 0 && s->rem_S != batch_size) {
            // keep one remainder size's graphs (as gs_step does)
            cudaStreamSynchronize(s->stream);
            for (int p = 0; p < 2; ++p) {
                auto it = s->graphs.find(std::make_pair(s->rem_S, p));
                if (it == s->graphs.end()) continue;
                cudaGraphExecDestroy(it->second.exec);
                cudaGraphDestroy(it->second.graph);
                s->graphs.erase(it);
            }
        }
        if (r > 0) s->rem_S = r;
        const auto t0 = std::chrono::steady_clock::now();
        const int64_t built = s->stats.graphs_built;
        st = prepare_graphs(s, n_iters, batch_size);
        if (st != GS_OK) return st;
        if (s->stats.graphs_built != built)
            s->stats.last_build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (nb > 0) {
            st = launch_graphs(s, batch_size, nb);
            if (st != GS_OK) return st;
        }
        if (r > 0) {
            st = launch_graphs(s, r, 1);
            if (st != GS_OK) return st;
        }
    }
    s->time += n_iters;
    s->stats.iterations += n_iters;
    return GS_OK;
}

gs_status gs_slab_set_time(gs_slab* s, int64_t n) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    if (n < 0) return sfail(s, GS_ERR_INVALID_ARG, "time must be >= 0");
    for (int k = 0; k < s->K; ++k) {
        gs_status st = gs_set_time(s->ctx[k], n);
        if (st != GS_OK) return from_slab(s, st, k);
    }
    s->time = n;
    return GS_OK;
}

gs_status gs_slab_sync(gs_slab* s) {
    if (!s) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set");
    GS_SCUDA(s, cudaStreamSynchronize(s->stream));
    GS_SCUDA(s, cudaGetLastError());
    return GS_OK;
}

gs_status gs_slab_get_stats(const gs_slab* s, gs_stats* out) {
    if (!s || !out) return global_fail(GS_ERR_INVALID_ARG, "NULL slab set or output pointer");
    *out = s->stats;
    return GS_OK;
}

}  // extern "C"
