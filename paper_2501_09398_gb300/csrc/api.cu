// C ABI of graphstep: contexts, field binding, per-step launches and the
// iteration-batch graph unroller (the paper's Sec. III-A, Listings 1-3).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

using namespace gs;

namespace {

thread_local std::string g_create_error;

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
    // Device-loop graphs only: the node that sets the trip count, and the
    // trip count it currently holds.
    cudaGraphNode_t init_node = nullptr;
    unsigned long long trip = 0;
};

// Device-side loop control of the while-node graphs.  The parent graph runs
// loop_init once (remaining = trip) and then the conditional node; the last
// node of the body runs loop_ctl, which counts one trip off and keeps the
// condition set while trips remain.  loop_ctl ends the loop on any value
// <= 1, so the loop stops after at most the stored count whatever it holds.
__global__ void loop_init_kernel(unsigned long long* remaining, unsigned long long trip) { *remaining = trip; }

__global__ void loop_ctl_kernel(cudaGraphConditionalHandle h, unsigned long long* remaining) {
    const unsigned long long left = *remaining;
    if (left <= 1) {
        *remaining = 0;
        cudaGraphSetConditional(h, 0u);
    } else {
        *remaining = left - 1;
        cudaGraphSetConditional(h, 1u);
    }
}

}  // namespace

struct gs_ctx {
    gs_kind kind;
    int64_t nx, ny, nz;
    gs_dtype dt;
    gs_bc bc;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    gs_heat_coeffs hc{0.5f, 0.1f, 0.1f, 0.01f, 0.05f, 80.0f};
    gs_fdtd_params fp{};
    float scale = 1.0f;
    gs_plan plan{};
    void* ptr[12] = {};
    int64_t pitch[12] = {};
    int parity = 0;
    int64_t time = 0;
    long long* d_counter = nullptr;
    unsigned long long* d_loop = nullptr;  // trips left of the device loop
    std::vector<gs_medium> media;           // FDTD media table (empty: vacuum)
    std::vector<float2> h_med;              // coefficients as uploaded
    float2* d_med = nullptr;                // [256] (da, db) | [256] (ca, cb)
    float* staging = nullptr;
    size_t staging_bytes = 0;
    // FDTD fused plan: the second set of the six components (library-owned,
    // component c at fused_set + c * fused_stride bytes) and the fused
    // launches reading set A (the bound fields) / set B (this one)
    char* fused_set = nullptr;
    size_t fused_stride = 0;
    LaunchDesc fdesc[2];
    // Launch descriptors, valid while descs_ok: thermal [0]=depth 1,
    // [1]=depth t, each per parity; FDTD [0][0]=H, [0][1]=E.
    LaunchDesc desc[2][2];
    bool descs_ok = false;
    std::map<std::pair<int64_t, int>, GraphEntry> graphs;
    std::map<std::pair<int64_t, int>, GraphEntry> loops;  // device-loop graphs
    int64_t built_S = 0;
    int64_t rem_S = 0;  // size of the peeled remainder graphs kept from gs_step (0: none)
    gs_stats stats{};
    std::string err;
};

// ------------------------------------------------------------ helpers ----

namespace {

gs_status fail(gs_ctx* c, gs_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

gs_status cuda_fail(gs_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA, m);
}

#define GS_CUDA(ctx, call)                                        \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

int vec_elems(gs_dtype dt) { return dt == GS_F32 ? 4 : 8; }
constexpr int kTemporalThreads = 256;  // threads of a temporally blocked tile
size_t elem_bytes(gs_dtype dt) { return dt == GS_F32 ? 4 : 2; }
bool is_heat(const gs_ctx* c) { return c->kind == GS_HEAT2D || c->kind == GS_HEAT3D; }
bool is_skel(const gs_ctx* c) { return c->kind == GS_SKELETON; }

// Dense row width, row count and element count of a field.
bool field_shape(const gs_ctx* c, int id, int64_t* width, int64_t* rows) {
    if (is_heat(c)) {
        if (id == GS_FIELD_T0 || id == GS_FIELD_T1) {
            *width = c->nx;
            *rows = c->ny * c->nz;
            return true;
        }
        if (id == GS_FIELD_P) {
            *width = c->nx;
            *rows = c->ny;
            return true;
        }
        return false;
    }
    if (is_skel(c)) {
        if (id != GS_FIELD_X) return false;
        *width = c->nx;
        *rows = 1;
        return true;
    }
    if ((id >= GS_FIELD_EX && id <= GS_FIELD_HZ) || id == GS_FIELD_MAT) {
        *width = c->nx + 1;
        *rows = (c->nx + 1) * (c->nz + 1);  // nz == nx except in a slab set's sub-domains
        return true;
    }
    return false;
}

int resolve(const gs_ctx* c, int id) {
    if (id == GS_FIELD_T) return c->parity ? GS_FIELD_T1 : GS_FIELD_T0;
    return id;
}

void destroy_graphs(gs_ctx* c) {
    for (auto* m : {&c->graphs, &c->loops}) {
        for (auto& kv : *m) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        m->clear();
    }
    c->built_S = 0;
    c->rem_S = 0;
}

// gs_step keeps the remainder graphs (both parities) of one remainder size
// only: a caller that varies n_iters would otherwise collect a graph of up to
// S-1 nodes per remainder it ever met.  Graphs of the size being launched as
// batches, or built by gs_graph_build, are left alone.
void drop_remainder(gs_ctx* c, int64_t keep_S) {
    const int64_t r = c->rem_S;
    if (r == 0 || r == keep_S || r == c->built_S) return;
    bool any = false;
    for (int p = 0; p < 2; ++p) any |= c->graphs.count(std::make_pair(r, p)) > 0;
    if (!any) return;
    cudaStreamSynchronize(c->stream);  // no launch of these graphs may still be pending
    for (int p = 0; p < 2; ++p) {
        auto it = c->graphs.find(std::make_pair(r, p));
        if (it == c->graphs.end()) continue;
        cudaGraphExecDestroy(it->second.exec);
        cudaGraphDestroy(it->second.graph);
        c->graphs.erase(it);
    }
}

void invalidate(gs_ctx* c) {
    destroy_graphs(c);
    c->descs_ok = false;
}

gs_plan default_plan(const gs_ctx* c) {
    gs_plan p{};
    if (is_skel(c)) {
        p.block_x = 256;
        p.rows = 1;
        p.temporal_depth = 1;
        return p;
    }
    if (c->kind == GS_FDTD3D) {
        p.block_x = 32;
        while (p.block_x * vec_elems(c->dt) < c->nx + 1 && p.block_x < 128) p.block_x += 32;
        p.rows = 4;  // COLUMN: j rows per block (k planes per block for MARCH)
        p.temporal_depth = 1;
        p.kernel = GS_KERNEL_COLUMN;
    } else {
        // the column kernel (measured fastest at depth 1 for 2D, thin stacks
        // and, in 8-plane chunks, deep stacks); rows = warps per block
        // stacked in y
        const bool small = c->nx * c->ny * c->nz <= (1 << 22);
        const bool deep = c->kind == GS_HEAT3D && c->nz > kColumnMaxNz;
        p.block_x = 64;
        p.rows = (small || deep) ? 4 : 8;
        p.tile_x = c->kind == GS_HEAT2D ? 64 : 32;
        p.tile_y = 32;
        p.temporal_depth = 1;
        p.kernel = GS_KERNEL_COLUMN;
    }
    return p;
}

gs_status validate_plan(gs_ctx* c, gs_plan* p) {
    const gs_plan d = default_plan(c);
    const bool block_x_given = p->block_x != 0;
    if (p->block_x == 0) p->block_x = d.block_x;
    if (p->rows == 0) p->rows = d.rows;
    if (p->tile_x == 0) p->tile_x = d.tile_x;
    if (p->tile_y == 0) p->tile_y = d.tile_y;
    if (p->temporal_depth == 0) p->temporal_depth = 1;
    if (p->graph_loop != 0 && p->graph_loop != 1) return fail(c, GS_ERR_INVALID_ARG, "plan.graph_loop must be 0 or 1");
    if (p->traverse < GS_TRAVERSE_AUTO || p->traverse > GS_TRAVERSE_ALTERNATE)
        return fail(c, GS_ERR_INVALID_ARG, "plan.traverse must be a gs_traverse value");
    if (p->graph_loop && p->device_launch)
        return fail(c, GS_ERR_UNSUPPORTED, "a device-launch graph cannot hold the conditional node of plan.graph_loop");
    if (p->block_x < 32 || p->block_x > 1024 || p->block_x % 32)
        return fail(c, GS_ERR_INVALID_ARG, "plan.block_x must be a multiple of 32 in [32, 1024]");
    if (p->rows < 1) return fail(c, GS_ERR_INVALID_ARG, "plan.rows must be >= 1");
    if ((c->kind == GS_FDTD3D || is_skel(c)) && p->block_x > 256)
        return fail(c, GS_ERR_INVALID_ARG, "FDTD / skeleton: plan.block_x must be <= 256");
    if (is_skel(c)) {
        if (p->temporal_depth > 1) return fail(c, GS_ERR_UNSUPPORTED, "the skeleton kernel has no temporal blocking");
        if (p->use_pdl != 0 && p->use_pdl != 1) return fail(c, GS_ERR_INVALID_ARG, "plan.use_pdl must be 0 or 1");
        if (p->device_launch != 0 && p->device_launch != 1)
            return fail(c, GS_ERR_INVALID_ARG, "plan.device_launch must be 0 or 1");
        if (p->use_pdl && p->device_launch)
            return fail(c, GS_ERR_INVALID_ARG, "plan.use_pdl and plan.device_launch cannot be combined");
        p->kernel = GS_KERNEL_AUTO;
        return GS_OK;
    }
    if (c->kind != GS_FDTD3D && p->block_x > 512)
        return fail(c, GS_ERR_INVALID_ARG, "thermal: plan.block_x must be <= 512");
    if (p->use_pdl != 0 && p->use_pdl != 1) return fail(c, GS_ERR_INVALID_ARG, "plan.use_pdl must be 0 or 1");
    if (p->device_launch != 0 && p->device_launch != 1)
        return fail(c, GS_ERR_INVALID_ARG, "plan.device_launch must be 0 or 1");
    if (p->use_pdl && p->device_launch)
        return fail(c, GS_ERR_INVALID_ARG, "plan.use_pdl and plan.device_launch cannot be combined");
    const int t = p->temporal_depth;
    if (t != 1 && t != 2 && t != 4) return fail(c, GS_ERR_INVALID_ARG, "plan.temporal_depth must be 1, 2 or 4");
    if (c->kind == GS_FDTD3D && t != 1)
        return fail(c, GS_ERR_UNSUPPORTED, "temporal blocking is provided for the thermal stencils only");
    if (p->kernel < GS_KERNEL_AUTO || p->kernel > GS_KERNEL_STREAM)
        return fail(c, GS_ERR_INVALID_ARG, "plan.kernel must be a gs_kernel value");
    if (c->kind == GS_FDTD3D) {
        if (p->kernel == GS_KERNEL_AUTO) p->kernel = GS_KERNEL_COLUMN;
        if (p->kernel != GS_KERNEL_COLUMN && p->kernel != GS_KERNEL_MARCH && p->kernel != GS_KERNEL_FUSED)
            return fail(c, GS_ERR_INVALID_ARG, "FDTD kernels: GS_KERNEL_COLUMN, GS_KERNEL_MARCH or GS_KERNEL_FUSED");
        if (p->kernel == GS_KERNEL_FUSED && (p->tile_y < 0 || p->tile_y > (1 << 20)))
            return fail(c, GS_ERR_INVALID_ARG, "FDTD FUSED: plan.tile_y (k planes a block marches; 0: none) must be in [0, 2^20]");
    } else if (p->kernel == GS_KERNEL_FUSED) {
        return fail(c, GS_ERR_INVALID_ARG, "GS_KERNEL_FUSED is an FDTD kernel");
    }
    if (p->kernel == GS_KERNEL_STREAM) {
        if (c->kind != GS_HEAT3D) return fail(c, GS_ERR_INVALID_ARG, "the STREAM kernel runs 3D thermal stacks only");
        if (t != 2) return fail(c, GS_ERR_INVALID_ARG, "the STREAM kernel runs temporal depth 2 only");
        if (p->block_x != 256 && p->block_x != 512)
            return fail(c, GS_ERR_INVALID_ARG, "the STREAM kernel takes plan.block_x 256 or 512");
        if (p->tile_y < 1 || p->tile_y > (1 << 20))
            return fail(c, GS_ERR_INVALID_ARG, "plan.tile_y (planes a block marches) must be in [1, 2^20]");
    }
    const bool wave_ok = (c->kind == GS_HEAT2D) || (c->nz <= kWaveMaxNz);
    if (is_heat(c) && p->kernel == GS_KERNEL_AUTO) {
        if (t == 2 && !wave_ok && (!block_x_given || p->block_x == 256 || p->block_x == 512)) {
            // deep stacks at depth 2: the planes streamed through shared memory
            p->kernel = GS_KERNEL_STREAM;
            if (!block_x_given) p->block_x = 256;
        } else {
            p->kernel = (t == 1 || c->kind == GS_HEAT2D || c->nz <= kColumnMaxNz || (t == 2 && !wave_ok))
                            ? GS_KERNEL_COLUMN
                            : (wave_ok ? GS_KERNEL_WAVE : GS_KERNEL_TILE);
        }
    }
    if (p->kernel == GS_KERNEL_MARCH && t != 1)
        return fail(c, GS_ERR_INVALID_ARG, "the MARCH kernel runs depth 1 only");
    if (p->kernel == GS_KERNEL_TILE && t == 1)
        return fail(c, GS_ERR_INVALID_ARG, "the TILE kernel runs depth 2 or 4 only");
    if (p->kernel == GS_KERNEL_COLUMN_SMEM && t != 1)
        return fail(c, GS_ERR_INVALID_ARG, "the COLUMN_SMEM kernel runs depth 1 only");
    if (p->kernel == GS_KERNEL_COLUMN && t == 4 && c->kind == GS_HEAT3D && c->nz > kColumnMaxNz)
        return fail(c, GS_ERR_UNSUPPORTED, "the COLUMN kernel runs depth 4 in 2D and for nz <= 8 only");
    if (p->kernel == GS_KERNEL_COLUMN && t == 2 && c->kind == GS_HEAT3D && c->nz > kColumnMaxNz &&
        (p->tile_y < 1 || p->tile_y > (1 << 20)))
        return fail(c, GS_ERR_INVALID_ARG, "plan.tile_y (planes a block marches) must be in [1, 2^20]");
    if (p->kernel == GS_KERNEL_COLUMN_SMEM && c->kind == GS_HEAT3D && c->nz > kColumnMaxNz)
        return fail(c, GS_ERR_UNSUPPORTED, "the COLUMN_SMEM kernel needs nz <= 8");
    if (p->kernel == GS_KERNEL_WAVE && !wave_ok)
        return fail(c, GS_ERR_UNSUPPORTED, "the WAVE kernel needs nz <= 16 (all planes in one block)");
    if (p->kernel == GS_KERNEL_WAVE && heat_wave_smem(c->kind == GS_HEAT3D ? (int)c->nz : 0, t, vec_elems(c->dt)) > 227 * 1024)
        return fail(c, GS_ERR_UNSUPPORTED, "WAVE kernel shared memory too large");
    if (t > 1 && p->kernel == GS_KERNEL_TILE) {
        if (p->tile_x < 1 || p->tile_y < 1 || p->tile_x > 4096 || p->tile_y > 4096)
            return fail(c, GS_ERR_INVALID_ARG, "plan.tile_x/tile_y must be in [1, 4096]");
        const size_t sm = heat_temporal_smem(c->kind == GS_HEAT3D ? (int)c->nz : 1, p->tile_x, p->tile_y, t);
        if (sm > 227 * 1024)
            return fail(c, GS_ERR_UNSUPPORTED, "temporal tile needs " + std::to_string(sm) +
                                                   " bytes of shared memory (limit 232448)");
    }
    if (c->kind == GS_HEAT3D && p->kernel == GS_KERNEL_MARCH) {
        const int zb = (int)std::min<int64_t>(std::min<int64_t>(c->nz, 16), std::max(1, 512 / p->block_x));
        if ((size_t)2 * (zb + 2) * p->block_x * vec_elems(c->dt) * 4 > 227 * 1024)
            return fail(c, GS_ERR_UNSUPPORTED, "3D depth-1 block needs too much shared memory");
    }
    return GS_OK;
}

gs_status require_fields(gs_ctx* c) {
    if (is_skel(c)) {
        if (!c->ptr[GS_FIELD_X]) return fail(c, GS_ERR_STATE, "field X must be bound before stepping");
        return GS_OK;
    }
    if (is_heat(c)) {
        if (!c->ptr[GS_FIELD_T0] || !c->ptr[GS_FIELD_T1] || !c->ptr[GS_FIELD_P])
            return fail(c, GS_ERR_STATE, "fields T0, T1 and P must be bound before stepping");
        if (c->pitch[GS_FIELD_T0] != c->pitch[GS_FIELD_T1])
            return fail(c, GS_ERR_STATE, "T0 and T1 must have the same pitch");
    } else {
        for (int f = GS_FIELD_EX; f <= GS_FIELD_HZ; ++f)
            if (!c->ptr[f]) return fail(c, GS_ERR_STATE, "all six FDTD components must be bound before stepping");
        for (int f = GS_FIELD_EY; f <= GS_FIELD_HZ; ++f)
            if (c->pitch[f] != c->pitch[GS_FIELD_EX])
                return fail(c, GS_ERR_STATE, "all six FDTD components must have the same pitch");
        if (!c->media.empty()) {
            if (!c->ptr[GS_FIELD_MAT]) return fail(c, GS_ERR_STATE, "a media table is set: bind GS_FIELD_MAT");
            if (c->pitch[GS_FIELD_MAT] != c->pitch[GS_FIELD_EX])
                return fail(c, GS_ERR_STATE, "GS_FIELD_MAT must have the components' pitch (in elements)");
        }
    }
    return GS_OK;
}

// Coefficients of the media table at the current courant number, all 256
// ids (vacuum past the table), uploaded to the context's device table.
gs_status upload_media(gs_ctx* c) {
    const double s = c->fp.courant;
    c->h_med.assign(2 * GS_MAX_MEDIA, make_float2(1.0f, (float)s));
    for (size_t m = 0; m < c->media.size(); ++m) {
        const gs_medium& r = c->media[m];
        const double ae = (double)r.sigma * s / (2.0 * r.eps_r);
        const double ah = (double)r.sigma_m * s / (2.0 * r.mu_r);
        c->h_med[m] = make_float2((float)((1.0 - ah) / (1.0 + ah)), (float)((s / r.mu_r) / (1.0 + ah)));
        c->h_med[GS_MAX_MEDIA + m] = make_float2((float)((1.0 - ae) / (1.0 + ae)), (float)((s / r.eps_r) / (1.0 + ae)));
    }
    if (!c->d_med) GS_CUDA(c, gs_malloc(&c->d_med, 2 * GS_MAX_MEDIA * sizeof(float2)));
    GS_CUDA(c, cudaMemcpyAsync(c->d_med, c->h_med.data(), 2 * GS_MAX_MEDIA * sizeof(float2), cudaMemcpyHostToDevice,
                               c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

gs_status ensure_descs(gs_ctx* c) {
    if (c->descs_ok) return GS_OK;
    gs_status st = require_fields(c);
    if (st != GS_OK) return st;
    if (is_skel(c)) {
        SkeletonArgs a{c->ptr[GS_FIELD_X], (long long)c->nx, c->scale};
        cudaError_t e = skeleton_desc(c->dt, a, c->plan.block_x, &c->desc[0][0]);
        if (e != cudaSuccess) return cuda_fail(c, e, "skeleton kernel set-up");
        c->descs_ok = true;
        return GS_OK;
    }
    if (is_heat(c)) {
        HeatArgs a{};
        a.P = c->ptr[GS_FIELD_P];
        a.nx = (int)c->nx;
        a.ny = (int)c->ny;
        a.nz = (int)c->nz;
        a.rows = c->plan.rows;
        a.pitch = c->pitch[GS_FIELD_T0];
        a.plane = a.pitch * c->ny;
        a.p_pitch = c->pitch[GS_FIELD_P];
        a.tile_x = c->plan.tile_x;
        a.tile_y = c->plan.tile_y;
        a.c = HeatCoef{c->hc.k, c->hc.cx, c->hc.cy, c->hc.cz, c->hc.cz2, c->hc.t_amb};
        const int t = c->plan.temporal_depth;
        // one step reads T and P and writes T
        const double step_bytes =
            (double)ctx_elem_bytes(c) * ((double)a.pitch * c->ny * c->nz * 2 + (double)a.p_pitch * c->ny);
        const bool alt = traverse_alternates(c->plan.traverse, step_bytes);
        for (int par = 0; par < 2; ++par) {
            a.Tin = c->ptr[par ? GS_FIELD_T1 : GS_FIELD_T0];
            a.Tout = c->ptr[par ? GS_FIELD_T0 : GS_FIELD_T1];
            a.rev = (alt && par == 1) ? 1 : 0;
            // single-step launches (depth 1, and the peeled n mod t steps)
            const int v1 = (c->plan.kernel == GS_KERNEL_WAVE || c->plan.kernel == GS_KERNEL_COLUMN ||
                            c->plan.kernel == GS_KERNEL_COLUMN_SMEM)
                               ? c->plan.kernel
                               : (c->plan.kernel == GS_KERNEL_STREAM ? GS_KERNEL_COLUMN : GS_KERNEL_MARCH);
            cudaError_t e = heat_desc(c->kind, c->dt, c->bc, a, c->plan.block_x, 1, v1, &c->desc[0][par]);
            if (e != cudaSuccess) return cuda_fail(c, e, "thermal kernel set-up");
            if (t > 1) {
                const int bx = (c->plan.kernel == GS_KERNEL_TILE) ? kTemporalThreads : c->plan.block_x;
                e = heat_desc(c->kind, c->dt, c->bc, a, bx, t, c->plan.kernel, &c->desc[1][par]);
                if (e != cudaSuccess) return cuda_fail(c, e, "temporal kernel set-up");
            }
        }
    } else {
        FdtdArgs a{};
        for (int f = 0; f < 6; ++f) a.f[f] = c->ptr[GS_FIELD_EX + f];
        a.N = (int)c->nx;
        a.Nk = (int)c->nz;
        a.kc = c->plan.rows;
        a.pitch = c->pitch[GS_FIELD_EX];
        a.plane = a.pitch * (c->nx + 1);
        a.s = c->fp.courant;
        a.src_on = c->fp.src_on;
        a.si = (int)c->fp.src_i;
        a.sj = (int)c->fp.src_j;
        a.sk = (int)c->fp.src_k;
        a.amp = c->fp.src_amp;
        a.delay = c->fp.src_delay;
        a.width = c->fp.src_width;
        a.counter = c->d_counter;
        a.mat = nullptr;
        a.med = nullptr;
        const bool fused = (c->plan.kernel == GS_KERNEL_FUSED);
        if (!c->media.empty()) {
            if (c->plan.kernel != GS_KERNEL_COLUMN && !(fused && c->plan.tile_y >= 1))
                return fail(c, GS_ERR_UNSUPPORTED,
                            "FDTD media run on the COLUMN kernels or the FUSED march (plan.tile_y >= 1) only");
            gs_status ms = upload_media(c);
            if (ms != GS_OK) return ms;
            a.mat = static_cast<const unsigned char*>(c->ptr[GS_FIELD_MAT]);
            a.med = c->d_med;
        }
        // one half-step reads all six components (and the ids), writes three
        const double step_bytes = (double)ctx_elem_bytes(c) * 6.0 * (double)a.plane * (double)(c->nz + 1) +
                                  (a.mat ? (double)a.plane * (double)(c->nz + 1) : 0.0);
        // fused: the in-place pair (COLUMN) serves an odd last step
        const int split = fused ? (int)GS_KERNEL_COLUMN : c->plan.kernel;
        a.rev = 0;
        cudaError_t e = fdtd_desc(c->dt, false, a, c->plan.block_x, split, &c->desc[0][0]);
        a.rev = traverse_alternates(c->plan.traverse, step_bytes) ? 1 : 0;
        if (e == cudaSuccess) e = fdtd_desc(c->dt, true, a, c->plan.block_x, split, &c->desc[0][1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "FDTD kernel set-up");
        if (fused) {
            const size_t stride = (((size_t)a.plane * (size_t)(c->nz + 1) * ctx_elem_bytes(c)) + 255) / 256 * 256;
            if (c->fused_stride != stride) {
                if (c->fused_set) {
                    cudaStreamSynchronize(c->stream);
                    cudaFree(c->fused_set);
                    c->fused_set = nullptr;
                    c->fused_stride = 0;
                }
                GS_CUDA(c, gs_malloc(&c->fused_set, 6 * stride));
                c->fused_stride = stride;
            }
            FdtdArgs b = a;
            b.kmarch = c->plan.tile_y;
            for (int f = 0; f < 6; ++f) b.g[f] = c->fused_set + (size_t)f * stride;
            b.rev = 0;
            e = fdtd_desc(c->dt, false, b, c->plan.block_x, GS_KERNEL_FUSED, &c->fdesc[0]);
            for (int f = 0; f < 6; ++f) std::swap(b.f[f], b.g[f]);
            b.rev = traverse_alternates(c->plan.traverse, step_bytes) ? 1 : 0;
            if (e == cudaSuccess) e = fdtd_desc(c->dt, false, b, c->plan.block_x, GS_KERNEL_FUSED, &c->fdesc[1]);
            if (e != cudaSuccess) return cuda_fail(c, e, "FDTD fused kernel set-up");
        }
    }
    c->descs_ok = true;
    return GS_OK;
}

// The kernel sequence of n iterations starting at buffer parity p, in
// order.  Thermal: n/t launches of depth t, then n%t of depth 1 (each flips
// the parity).  FDTD: H, E per iteration.
template <typename F>
void for_each_launch(gs_ctx* c, int64_t n, int p, F&& f) {
    if (is_skel(c)) {
        for (int64_t i = 0; i < n; ++i) f(c->desc[0][0]);
        return;
    }
    if (is_heat(c)) {
        const int t = c->plan.temporal_depth;
        const int64_t q = (t > 1) ? n / t : 0;
        const int64_t r = n - q * t;
        for (int64_t i = 0; i < q; ++i) { f(c->desc[1][p]); p ^= 1; }
        for (int64_t i = 0; i < r; ++i) { f(c->desc[0][p]); p ^= 1; }
    } else if (c->plan.kernel == GS_KERNEL_FUSED) {
        // pairs of fused steps (A -> B, B -> A), so the state ends in A;
        // an odd last step runs the in-place H and E launches
        for (int64_t i = 0; i < n / 2; ++i) { f(c->fdesc[0]); f(c->fdesc[1]); }
        if (n & 1) { f(c->desc[0][0]); f(c->desc[0][1]); }
    } else {
        for (int64_t i = 0; i < n; ++i) { f(c->desc[0][0]); f(c->desc[0][1]); }
    }
}

int64_t launches_for(const gs_ctx* c, int64_t n) {
    if (is_skel(c)) return n;
    if (!is_heat(c)) return c->plan.kernel == GS_KERNEL_FUSED ? n + (n & 1) : 2 * n;
    const int t = c->plan.temporal_depth;
    const int64_t q = (t > 1) ? n / t : 0;
    return q + (n - q * t);
}

int flip_of(const gs_ctx* c, int64_t n) { return is_heat(c) ? (int)(launches_for(c, n) & 1) : 0; }

cudaError_t launch_one(gs_ctx* c, LaunchDesc& d) {
    void* args[1] = {d.arg_ptr()};
    if (!c->plan.use_pdl) return cudaLaunchKernel(d.func, d.grid, d.block, args, d.smem, c->stream);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = d.grid;
    cfg.blockDim = d.block;
    cfg.dynamicSmemBytes = d.smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, d.func, args);
}

// Append the kernel nodes of S iterations from parity p to g as a linear
// chain after *prev (none if NULL), with programmatic edges when the plan
// asks for PDL.  *prev becomes the last node added.
cudaError_t add_chain(gs_ctx* c, cudaGraph_t g, int64_t S, int p, cudaGraphNode_t* prev, int64_t* nodes) {
    cudaError_t err = cudaSuccess;
    cudaGraphEdgeData edge{};
    edge.from_port = cudaGraphKernelNodePortProgrammatic;
    edge.to_port = 0;
    edge.type = cudaGraphDependencyTypeProgrammatic;
    for_each_launch(c, S, p, [&](LaunchDesc& d) {
        if (err != cudaSuccess) return;
        cudaKernelNodeParams np{};
        void* args[1] = {d.arg_ptr()};
        np.func = const_cast<void*>(d.func);
        np.gridDim = d.grid;
        np.blockDim = d.block;
        np.sharedMemBytes = (unsigned)d.smem;
        np.kernelParams = args;
        np.extra = nullptr;
        cudaGraphNode_t node;
        if (c->plan.use_pdl && *prev) {
            err = gs_graph_add_kernel_node(&node, g, nullptr, 0, &np);
            if (err == cudaSuccess) err = cudaGraphAddDependencies(g, prev, &node, &edge, 1);
        } else {
            err = gs_graph_add_kernel_node(&node, g, *prev ? prev : nullptr, *prev ? 1 : 0, &np);
        }
        *prev = node;
        ++*nodes;
    });
    return err;
}

gs_status instantiate(gs_ctx* c, cudaGraph_t g, GraphEntry* out) {
    cudaGraphExec_t exec = nullptr;
    const unsigned long long flags = c->plan.device_launch ? cudaGraphInstantiateFlagDeviceLaunch : 0;
    cudaError_t err = cudaGraphInstantiateWithFlags(&exec, g, flags);
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, err, "cudaGraphInstantiateWithFlags");
    }
    err = cudaGraphUpload(exec, c->stream);
    if (err != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
        return cuda_fail(c, err, "cudaGraphUpload");
    }
    out->graph = g;
    out->exec = exec;
    c->stats.graphs_built += 1;
    return GS_OK;
}

// Build one executable graph of S iterations from parity p: the paper's
// manual creation of a linear chain (Listing 3, "Building"), optionally
// with programmatic edges, then instantiate and upload.
gs_status build_graph(gs_ctx* c, int64_t S, int p, GraphEntry* out) {
    cudaGraph_t g = nullptr;
    GS_CUDA(c, cudaGraphCreate(&g, 0));
    cudaGraphNode_t prev = nullptr;
    int64_t nodes = 0;
    cudaError_t err = add_chain(c, g, S, p, &prev, &nodes);
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, err, "cudaGraphAddKernelNode");
    }
    out->nodes = nodes;
    return instantiate(c, g, out);
}

// Build the device-loop graph of batches of S from parity p: loop_init,
// then a while node whose body is one batch (two when a batch flips the
// parity, so every trip starts at p) followed by loop_ctl.  One launch runs
// `trip` bodies with no host launch between them; the trip count is a
// parameter of the init node, changed in the executable graph per launch.
gs_status build_loop(gs_ctx* c, int64_t S, int p, GraphEntry* out) {
    if (!c->d_loop) GS_CUDA(c, gs_malloc(&c->d_loop, sizeof(unsigned long long)));
    cudaGraph_t g = nullptr;
    GS_CUDA(c, cudaGraphCreate(&g, 0));
    cudaError_t err = cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNode_t init = nullptr, loop = nullptr;
    unsigned long long trip = 1;
    void* init_args[2] = {&c->d_loop, &trip};
    cudaKernelNodeParams ip{};
    ip.func = (void*)loop_init_kernel;
    ip.gridDim = dim3(1);
    ip.blockDim = dim3(1);
    ip.kernelParams = init_args;
    err = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (err == cudaSuccess) err = gs_graph_add_kernel_node(&init, g, nullptr, 0, &ip);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (err == cudaSuccess) err = cudaGraphAddNode(&loop, g, &init, nullptr, 1, &cp);
    int64_t nodes = 0;
    if (err == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t prev = nullptr;
        const int fl = flip_of(c, S);
        err = add_chain(c, body, S, p, &prev, &nodes);
        if (err == cudaSuccess && fl) err = add_chain(c, body, S, p ^ 1, &prev, &nodes);
        void* ctl_args[2] = {&h, &c->d_loop};
        cudaKernelNodeParams kp{};
        kp.func = (void*)loop_ctl_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = ctl_args;
        cudaGraphNode_t ctl;
        if (err == cudaSuccess) err = gs_graph_add_kernel_node(&ctl, body, &prev, 1, &kp);
    }
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, err, "device-loop graph construction");
    }
    out->nodes = nodes;
    out->init_node = init;
    out->trip = trip;
    return instantiate(c, g, out);
}

gs_status ensure_graph(gs_ctx* c, int64_t S, int p, GraphEntry** out) {
    auto key = std::make_pair(S, p);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        GraphEntry e;
        gs_status st = build_graph(c, S, p, &e);
        if (st != GS_OK) return st;
        it = c->graphs.emplace(key, e).first;
    }
    *out = &it->second;
    return GS_OK;
}

gs_status ensure_loop(gs_ctx* c, int64_t S, int p, GraphEntry** out) {
    auto key = std::make_pair(S, p);
    auto it = c->loops.find(key);
    if (it == c->loops.end()) {
        GraphEntry e;
        gs_status st = build_loop(c, S, p, &e);
        if (st != GS_OK) return st;
        it = c->loops.emplace(key, e).first;
    }
    *out = &it->second;
    return GS_OK;
}

gs_status launch_graphs(gs_ctx* c, int64_t S, int64_t count);

// Run `count` batches of S with the device loop: one launch of the loop
// graph for the whole bodies (count, or count/2 when a batch flips the
// parity), then the odd batch, if any, as a plain batch graph.
gs_status launch_loop(gs_ctx* c, int64_t S, int64_t count) {
    const int fl = flip_of(c, S);
    const int64_t trips = fl ? count / 2 : count;
    if (trips > 0) {
        GraphEntry* e;
        gs_status st = ensure_loop(c, S, c->parity, &e);
        if (st != GS_OK) return st;
        if (e->trip != (unsigned long long)trips) {
            unsigned long long trip = (unsigned long long)trips;
            void* args[2] = {&c->d_loop, &trip};
            cudaKernelNodeParams ip{};
            ip.func = (void*)loop_init_kernel;
            ip.gridDim = dim3(1);
            ip.blockDim = dim3(1);
            ip.kernelParams = args;
            GS_CUDA(c, cudaGraphExecKernelNodeSetParams(e->exec, e->init_node, &ip));
            e->trip = trip;
        }
        GS_CUDA(c, cudaGraphLaunch(e->exec, c->stream));
        c->stats.graph_launches += 1;
    }
    if (fl && (count & 1)) return launch_graphs(c, S, 1);
    return GS_OK;
}

// Build (if missing) every graph gs_step(n, S) launches from the current
// parity, before its first launch: a failed build then leaves the context as
// it was (no batch launched, parity and time unchanged).
gs_status prepare_step_graphs(gs_ctx* c, int64_t n, int64_t S) {
    const int64_t nb = n / S, r = n - nb * S;
    const int fl = flip_of(c, S);
    int p = c->parity;
    GraphEntry* e = nullptr;
    gs_status st = GS_OK;
    if (nb > 0) {
        if (c->plan.graph_loop) {
            if ((fl ? nb / 2 : nb) > 0) st = ensure_loop(c, S, p, &e);
            if (st == GS_OK && fl && (nb & 1)) st = ensure_graph(c, S, p, &e);
        } else {
            st = ensure_graph(c, S, p, &e);
            if (st == GS_OK && fl && nb > 1) st = ensure_graph(c, S, p ^ 1, &e);
        }
        if (st != GS_OK) return st;
        p ^= fl & (int)(nb & 1);
    }
    if (r > 0) st = ensure_graph(c, r, p, &e);
    return st;
}

// `count` batches of S: graph launches (Listing 3) or the device loop.
gs_status run_batches(gs_ctx* c, int64_t S, int64_t count) {
    return c->plan.graph_loop ? launch_loop(c, S, count) : launch_graphs(c, S, count);
}

gs_status launch_graphs(gs_ctx* c, int64_t S, int64_t count) {
    const int fl = flip_of(c, S);
    for (int64_t i = 0; i < count; ++i) {
        GraphEntry* e;
        gs_status st = ensure_graph(c, S, c->parity, &e);
        if (st != GS_OK) return st;
        GS_CUDA(c, cudaGraphLaunch(e->exec, c->stream));
        c->stats.graph_launches += 1;
        c->parity ^= fl;
    }
    return GS_OK;
}

gs_status ensure_staging(gs_ctx* c, size_t bytes) {
    if (c->staging_bytes >= bytes) return GS_OK;
    if (c->staging) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->staging);
        c->staging = nullptr;
        c->staging_bytes = 0;
    }
    GS_CUDA(c, gs_malloc(&c->staging, bytes));
    c->staging_bytes = bytes;
    return GS_OK;
}

bool finite_all(const float* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

namespace gs {
void ctx_field(const gs_ctx* c, int id, void** ptr, int64_t* pitch) {
    *ptr = c->ptr[id];
    *pitch = c->pitch[id];
}
bool ctx_shape(const gs_ctx* c, int id, int64_t* width, int64_t* rows) { return field_shape(c, id, width, rows); }
size_t ctx_elem_bytes(const gs_ctx* c) { return elem_bytes(c->dt); }
bool ctx_is_heat(const gs_ctx* c) { return is_heat(c); }
bool ctx_is_skel(const gs_ctx* c) { return is_skel(c); }
cudaStream_t ctx_stream(const gs_ctx* c) { return c->stream; }
gs_status ctx_fail(gs_ctx* c, gs_status s, const std::string& msg) { return fail(c, s, msg); }
gs_status global_fail(gs_status s, const std::string& msg) { return fail(nullptr, s, msg); }

namespace inject {
// Armed injection: the call kind and how many more calls of it succeed
// before the failing one (-1: disarmed).
std::atomic<int> g_inject_kind{GS_INJECT_NONE};
std::atomic<long long> g_inject_left{-1};

bool injected(int kind) {
    if (g_inject_kind.load() != kind) return false;
    const long long left = g_inject_left.fetch_sub(1);
    if (left > 0) return false;
    if (left == 0) {  // this call fails, then the injection is disarmed
        g_inject_kind.store(GS_INJECT_NONE);
        return true;
    }
    return false;
}
}  // namespace inject

cudaError_t gs_malloc_raw(void** p, size_t bytes) {
    if (inject::injected(GS_INJECT_MALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t gs_graph_add_kernel_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t n,
                                     const cudaKernelNodeParams* params) {
    if (inject::injected(GS_INJECT_GRAPH_NODE)) return cudaErrorInvalidValue;
    return cudaGraphAddKernelNode(node, g, deps, n, params);
}

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

size_t device_l2_bytes() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return 0;
    return n > 0 ? (size_t)n : 0;
}

bool traverse_alternates(int mode, double step_bytes) {
    if (mode == GS_TRAVERSE_FORWARD) return false;
    if (mode == GS_TRAVERSE_ALTERNATE) return true;
    return step_bytes > 0.5 * (double)device_l2_bytes();
}
}  // namespace gs

// ------------------------------------------------------------- C ABI -----

namespace {

// The grid checks of gs_create: nullptr if (kind, sizes, storage, bc) make a
// valid context, else why not.
const char* grid_error(gs_kind kind, int64_t nx, int64_t ny, int64_t nz, gs_dtype storage, gs_bc bc,
                       bool fdtd_box = false) {
    if (kind != GS_HEAT2D && kind != GS_HEAT3D && kind != GS_FDTD3D && kind != GS_SKELETON) return "unknown kind";
    if (kind == GS_SKELETON && (ny != 1 || nz != 1 || nx < 1 || nx >= (int64_t(1) << 31)))
        return "GS_SKELETON needs ny == nz == 1 and 1 <= nx < 2^31";
    if (storage != GS_F32 && storage != GS_BF16 && storage != GS_F16) return "unknown storage dtype";
    const int64_t lim = int64_t(1) << 20;
    if (kind != GS_SKELETON && (nx < 1 || ny < 1 || nz < 1 || nx > lim || ny > lim || nz > lim))
        return "grid sizes must be in [1, 2^20]";
    if (kind == GS_HEAT2D && nz != 1) return "GS_HEAT2D needs nz == 1";
    if (kind == GS_FDTD3D && (nx != ny || (ny != nz && !fdtd_box))) return "GS_FDTD3D needs a cubic grid (nx == ny == nz)";
    const int64_t w = (kind == GS_FDTD3D) ? nx + 1 : nx;
    const int64_t rows = (kind == GS_FDTD3D) ? (nx + 1) * (nz + 1) : ny * nz;
    if (kind != GS_SKELETON && (double)(w + 8) * (double)rows >= 2147483647.0)
        return "field too large (needs >= 2^31 elements)";
    if (kind == GS_FDTD3D && bc != GS_BC_PEC) return "GS_FDTD3D needs GS_BC_PEC";
    if ((kind == GS_HEAT2D || kind == GS_HEAT3D) && bc != GS_BC_CLAMP && bc != GS_BC_DIRICHLET0)
        return "thermal kinds need GS_BC_CLAMP or GS_BC_DIRICHLET0";
    return nullptr;
}

}  // namespace

extern "C" {

int gs_version(void) { return 100; }

const char* gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "GS_OK";
        case GS_ERR_INVALID_ARG: return "GS_ERR_INVALID_ARG";
        case GS_ERR_CUDA: return "GS_ERR_CUDA";
        case GS_ERR_OOM: return "GS_ERR_OOM";
        case GS_ERR_STATE: return "GS_ERR_STATE";
        case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
        case GS_ERR_NUMERIC: return "GS_ERR_NUMERIC";
        case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
    }
    return "GS_ERR_UNKNOWN";
}

const char* gs_last_error(const gs_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

gs_status gs_debug_inject_failure(gs_inject call, int64_t after) {
    if (call == GS_INJECT_NONE) {
        gs::inject::g_inject_kind.store(GS_INJECT_NONE);
        gs::inject::g_inject_left.store(-1);
        return GS_OK;
    }
    if ((call != GS_INJECT_MALLOC && call != GS_INJECT_GRAPH_NODE) || after < 0)
        return fail(nullptr, GS_ERR_INVALID_ARG, "gs_debug_inject_failure: unknown call kind or after < 0");
    gs::inject::g_inject_kind.store(GS_INJECT_NONE);
    gs::inject::g_inject_left.store(after);
    gs::inject::g_inject_kind.store(call);
    return GS_OK;
}

gs_status gs_debug_owned_ranges(const gs_ctx* c, uint64_t* lo, uint64_t* hi, int32_t capacity, int32_t* n_out) {
    if (!c || !n_out || capacity < 0 || (capacity > 0 && (!lo || !hi)))
        return fail(nullptr, GS_ERR_INVALID_ARG, "gs_debug_owned_ranges: bad arguments");
    int32_t n = 0;
    if (c->fused_set) {
        if (n < capacity) {
            lo[n] = reinterpret_cast<uint64_t>(c->fused_set);
            hi[n] = lo[n] + 6 * c->fused_stride;
        }
        ++n;
    }
    *n_out = n;
    return GS_OK;
}

int gs_debug_checked_build(void) {
#ifdef GS_CHECKED
    return 1;
#else
    return 0;
#endif
}

gs_status gs_debug_check_ranges(const uint64_t* lo, const uint64_t* hi, int32_t n) {
    if (n < 0 || n > GS_CHECK_MAX_RANGES || (n > 0 && (!lo || !hi)))
        return fail(nullptr, GS_ERR_INVALID_ARG, "gs_debug_check_ranges: n in [0, 128] and both arrays needed");
    for (int32_t i = 0; i < n; ++i)
        if (lo[i] > hi[i]) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_debug_check_ranges: lo > hi");
    if (!gs_debug_checked_build()) return fail(nullptr, GS_ERR_UNSUPPORTED, "not a bounds-checked build");
    static_assert(sizeof(uint64_t) == sizeof(unsigned long long), "range words");
    const auto* l = reinterpret_cast<const unsigned long long*>(lo);
    const auto* h = reinterpret_cast<const unsigned long long*>(hi);
    cudaError_t e = gs::heat_check_set(l, h, n);
    if (e == cudaSuccess) e = gs::fdtd_check_set(l, h, n);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "gs_debug_check_ranges");
    return GS_OK;
}

gs_status gs_debug_check_read(uint64_t* refused, uint64_t* first) {
    if (!refused || !first) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_debug_check_read: NULL argument");
    if (!gs_debug_checked_build()) return fail(nullptr, GS_ERR_UNSUPPORTED, "not a bounds-checked build");
    unsigned long long b1 = 0, f1 = 0, b2 = 0, f2 = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = gs::heat_check_get(&b1, &f1);
    if (e == cudaSuccess) e = gs::fdtd_check_get(&b2, &f2);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "gs_debug_check_read");
    *refused = b1 + b2;
    *first = b1 ? f1 : f2;
    return GS_OK;
}

gs_status gs_wait_timeouts(uint64_t* count_out) {
    if (!count_out) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_wait_timeouts: NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "gs_wait_timeouts");
    const unsigned n = gs::heat_stream_timeouts_take();
    if (n == ~0u) return cuda_fail(nullptr, cudaGetLastError(), "gs_wait_timeouts: reading the count");
    *count_out = n;
    return GS_OK;
}

gs_status gs_debug_injection_pending(int32_t* pending) {
    if (!pending) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_debug_injection_pending: NULL argument");
    *pending = gs::inject::g_inject_kind.load() != GS_INJECT_NONE;
    return GS_OK;
}

gs_status gs_required_pitch(gs_dtype dtype, int64_t width, int64_t* pitch_out) {
    if (!pitch_out || width < 1 || (dtype != GS_F32 && dtype != GS_BF16 && dtype != GS_F16))
        return fail(nullptr, GS_ERR_INVALID_ARG, "gs_required_pitch: need width >= 1, a known dtype and pitch_out");
    const int64_t v = vec_elems(dtype);
    *pitch_out = (width + v - 1) / v * v;
    return GS_OK;
}

gs_status gs_create(gs_ctx** out, gs_kind kind, int64_t nx, int64_t ny, int64_t nz, gs_dtype storage, gs_bc bc,
                    void* stream) {
    return gs::ctx_create(out, kind, nx, ny, nz, storage, bc, stream, false);
}

}  // extern "C"

namespace gs {

// gs_create, and (fdtd_box) FDTD contexts of N x N x Nk cells for the
// sub-domains of a slab set.
gs_status ctx_create(gs_ctx** out, gs_kind kind, int64_t nx, int64_t ny, int64_t nz, gs_dtype storage, gs_bc bc,
                     void* stream, bool fdtd_box) {
    if (!out) return fail(nullptr, GS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (const char* why = grid_error(kind, nx, ny, nz, storage, bc, fdtd_box))
        return fail(nullptr, GS_ERR_INVALID_ARG, why);

    gs_ctx* c = new (std::nothrow) gs_ctx();
    if (!c) return fail(nullptr, GS_ERR_OOM, "host allocation failed");
    c->kind = kind;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->dt = storage;
    c->bc = bc;
    c->fp = gs_fdtd_params{0.5f, 0, nx / 2, nx / 2, nx / 2, 1.0f, 60.0f, 20.0f};
    c->plan = default_plan(c);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) {
        if (stream) {
            c->stream = static_cast<cudaStream_t>(stream);
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess && kind == GS_FDTD3D) {
        e = gs_malloc(&c->d_counter, sizeof(long long));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counter, 0, sizeof(long long), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        gs_status st = cuda_fail(nullptr, e, "context set-up");
        gs_destroy(c);
        return st;
    }
    *out = c;
    return GS_OK;
}

gs_status ctx_prepare(gs_ctx* c) { return ensure_descs(c); }

void ctx_launch_list(gs_ctx* c, int64_t n, int p, std::vector<LaunchDesc*>* out) {
    for_each_launch(c, n, p, [&](LaunchDesc& d) { out->push_back(&d); });
}

int ctx_flip(const gs_ctx* c, int64_t n) { return flip_of(c, n); }

void ctx_workload(const gs_ctx* c, gs_workload* w) {
    *w = gs_workload{};
    w->kind = c->kind;
    w->dtype = c->dt;
    w->nx = c->nx;
    w->ny = c->ny;
    w->nz = c->nz;
    w->n_iters = c->time;
}

bool ctx_has_media(const gs_ctx* c) { return c->kind == GS_FDTD3D && !c->media.empty(); }

cudaError_t ctx_launch(gs_ctx* c, LaunchDesc& d) { return launch_one(c, d); }

}  // namespace gs

extern "C" {

gs_status gs_destroy(gs_ctx* c) {
    if (!c) return GS_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    destroy_graphs(c);
    if (c->d_counter) cudaFree(c->d_counter);
    if (c->d_loop) cudaFree(c->d_loop);
    if (c->d_med) cudaFree(c->d_med);
    if (c->staging) cudaFree(c->staging);
    if (c->fused_set) cudaFree(c->fused_set);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return GS_OK;
}

gs_status gs_set_heat_coeffs(gs_ctx* c, const gs_heat_coeffs* hc) {
    if (!c || !hc) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    if (!is_heat(c)) return fail(c, GS_ERR_INVALID_ARG, "not a thermal context");
    if (!finite_all(&hc->k, 6)) return fail(c, GS_ERR_NUMERIC, "non-finite coefficient");
    c->hc = *hc;
    invalidate(c);
    return GS_OK;
}

gs_status gs_set_scale(gs_ctx* c, float scale) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    if (!is_skel(c)) return fail(c, GS_ERR_INVALID_ARG, "not a skeleton context");
    if (!std::isfinite(scale)) return fail(c, GS_ERR_NUMERIC, "non-finite scale");
    c->scale = scale;
    invalidate(c);
    return GS_OK;
}

gs_status gs_set_fdtd_params(gs_ctx* c, const gs_fdtd_params* p) {
    if (!c || !p) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    if (c->kind != GS_FDTD3D) return fail(c, GS_ERR_INVALID_ARG, "not an FDTD context");
    const float f[4] = {p->courant, p->src_amp, p->src_delay, p->src_width};
    if (!finite_all(f, 4)) return fail(c, GS_ERR_NUMERIC, "non-finite parameter");
    if (p->src_width == 0.0f) return fail(c, GS_ERR_INVALID_ARG, "src_width must be non-zero");
    if (p->src_on != 0 && p->src_on != 1) return fail(c, GS_ERR_INVALID_ARG, "src_on must be 0 or 1");
    const int64_t N = c->nx;
    if (p->src_i < 0 || p->src_j < 0 || p->src_k < 0 || p->src_i > N || p->src_j > N || p->src_k > c->nz)
        return fail(c, GS_ERR_INVALID_ARG, "source cell outside the (N+1)^3 arrays");
    c->fp = *p;
    invalidate(c);
    return GS_OK;
}

gs_status gs_set_fdtd_media(gs_ctx* c, const gs_medium* table, int32_t n) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    if (c->kind != GS_FDTD3D) return fail(c, GS_ERR_INVALID_ARG, "not an FDTD context");
    if (n < 0 || n > GS_MAX_MEDIA) return fail(c, GS_ERR_INVALID_ARG, "media table: 0 <= n <= 256 rows");
    if (n > 0 && !table) return fail(c, GS_ERR_INVALID_ARG, "NULL media table");
    for (int32_t m = 0; m < n; ++m) {
        const gs_medium& r = table[m];
        if (!finite_all(&r.eps_r, 4)) return fail(c, GS_ERR_NUMERIC, "media row " + std::to_string(m) + ": non-finite");
        if (!(r.eps_r > 0.f) || !(r.mu_r > 0.f) || r.sigma < 0.f || r.sigma_m < 0.f)
            return fail(c, GS_ERR_INVALID_ARG,
                        "media row " + std::to_string(m) + ": need eps_r > 0, mu_r > 0, sigma >= 0, sigma_m >= 0");
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->media.assign(table, table + n);
    invalidate(c);
    return GS_OK;
}

gs_status gs_upload_u8(gs_ctx* c, gs_field id, const uint8_t* host, int64_t n) {
    if (!c || !host) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    int64_t width, rows;
    if (id != GS_FIELD_MAT || !field_shape(c, id, &width, &rows))
        return fail(c, GS_ERR_INVALID_ARG, "gs_upload_u8 takes GS_FIELD_MAT of an FDTD context");
    if (!c->ptr[id]) return fail(c, GS_ERR_STATE, "field is not bound");
    if (n != width * rows)
        return fail(c, GS_ERR_INVALID_ARG, "n must equal the dense element count " + std::to_string(width * rows));
    GS_CUDA(c, cudaMemcpy2DAsync(c->ptr[id], c->pitch[id], host, width, width, rows, cudaMemcpyHostToDevice,
                                 c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

gs_status gs_set_plan(gs_ctx* c, const gs_plan* plan) {
    if (!c || !plan) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    gs_plan p = *plan;
    gs_status st = validate_plan(c, &p);
    if (st != GS_OK) return st;
    c->plan = p;
    invalidate(c);
    return GS_OK;
}

gs_status gs_plan_check(const gs_workload* w, const gs_plan* plan, gs_plan* resolved) {
    if (!w || !plan) return fail(nullptr, GS_ERR_INVALID_ARG, "gs_plan_check: NULL argument");
    const gs_kind kind = static_cast<gs_kind>(w->kind);
    const gs_bc bc = (kind == GS_FDTD3D) ? GS_BC_PEC : GS_BC_CLAMP;  // no plan rule depends on the thermal bc
    if (const char* why = grid_error(kind, w->nx, w->ny, w->nz, static_cast<gs_dtype>(w->dtype), bc))
        return fail(nullptr, GS_ERR_INVALID_ARG, std::string("gs_plan_check: ") + why);
    gs_ctx c;  // the grid only: no stream, fields or device memory
    c.kind = kind;
    c.nx = w->nx;
    c.ny = w->ny;
    c.nz = w->nz;
    c.dt = static_cast<gs_dtype>(w->dtype);
    c.bc = bc;
    gs_plan p = *plan;
    const gs_status st = validate_plan(&c, &p);
    if (st != GS_OK) return fail(nullptr, st, "gs_plan_check: " + c.err);
    if (resolved) *resolved = p;
    return GS_OK;
}

gs_status gs_get_plan(const gs_ctx* c, gs_plan* out) {
    if (!c || !out) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context or output pointer");
    *out = c->plan;
    return GS_OK;
}

gs_status gs_bind_field(gs_ctx* c, gs_field id, void* ptr, int64_t pitch) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    const int f = resolve(c, id);
    int64_t width, rows;
    if (f < 0 || f > GS_FIELD_MAT || f == GS_FIELD_T || !field_shape(c, f, &width, &rows))
        return fail(c, GS_ERR_INVALID_ARG, "field id not valid for this context kind");
    if (ptr) {
        if (reinterpret_cast<uintptr_t>(ptr) % 16)
            return fail(c, GS_ERR_INVALID_ARG, "field pointer must be 16-byte aligned");
        if (pitch < width || pitch % vec_elems(c->dt))
            return fail(c, GS_ERR_INVALID_ARG,
                        "pitch must be >= " + std::to_string(width) + " and a multiple of 16 bytes");
        cudaPointerAttributes attr;
        cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaPointerGetAttributes");
        if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
            return fail(c, GS_ERR_INVALID_ARG, "field pointer is not device memory");
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->ptr[f] = ptr;
    c->pitch[f] = ptr ? pitch : 0;
    invalidate(c);
    return GS_OK;
}

gs_status gs_upload(gs_ctx* c, gs_field id, const float* host, int64_t n) {
    if (!c || !host) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    const int f = resolve(c, id);
    int64_t width, rows;
    if (f < 0 || f > GS_FIELD_X || f == GS_FIELD_T || !field_shape(c, f, &width, &rows))
        return fail(c, GS_ERR_INVALID_ARG, "field id not valid for this context kind");
    if (!c->ptr[f]) return fail(c, GS_ERR_STATE, "field is not bound");
    if (n != width * rows)
        return fail(c, GS_ERR_INVALID_ARG, "n must equal the dense element count " + std::to_string(width * rows));
    if (c->dt == GS_F32) {
        GS_CUDA(c, cudaMemcpy2DAsync(c->ptr[f], c->pitch[f] * 4, host, width * 4, width * 4, rows,
                                     cudaMemcpyHostToDevice, c->stream));
    } else {
        gs_status st = ensure_staging(c, (size_t)n * sizeof(float));
        if (st != GS_OK) return st;
        GS_CUDA(c, cudaMemcpyAsync(c->staging, host, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        GS_CUDA(c, convert_to_storage(c->dt, c->staging, c->ptr[f], width, rows, c->pitch[f], c->stream));
    }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

gs_status gs_read_field(gs_ctx* c, gs_field id, float* host_out, int64_t n) {
    if (!c || !host_out) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    const int f = resolve(c, id);
    int64_t width, rows;
    if (f < 0 || f > GS_FIELD_X || f == GS_FIELD_T || !field_shape(c, f, &width, &rows))
        return fail(c, GS_ERR_INVALID_ARG, "field id not valid for this context kind");
    if (!c->ptr[f]) return fail(c, GS_ERR_STATE, "field is not bound");
    if (n != width * rows)
        return fail(c, GS_ERR_INVALID_ARG, "n must equal the dense element count " + std::to_string(width * rows));
    if (c->dt == GS_F32) {
        GS_CUDA(c, cudaMemcpy2DAsync(host_out, width * 4, c->ptr[f], c->pitch[f] * 4, width * 4, rows,
                                     cudaMemcpyDeviceToHost, c->stream));
    } else {
        gs_status st = ensure_staging(c, (size_t)n * sizeof(float));
        if (st != GS_OK) return st;
        GS_CUDA(c, convert_from_storage(c->dt, c->ptr[f], c->staging, width, rows, c->pitch[f], c->stream));
        GS_CUDA(c, cudaMemcpyAsync(host_out, c->staging, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

gs_status gs_get_parity(const gs_ctx* c, int32_t* out) {
    if (!c || !out) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context or output pointer");
    *out = c->parity;
    return GS_OK;
}

gs_status gs_set_parity(gs_ctx* c, int32_t parity) {
    if (!c || (parity != 0 && parity != 1)) return fail(c, GS_ERR_INVALID_ARG, "parity must be 0 or 1");
    if (!is_heat(c)) return fail(c, GS_ERR_INVALID_ARG, "parity applies to thermal contexts only");
    c->parity = parity;
    return GS_OK;
}

gs_status gs_set_time(gs_ctx* c, int64_t n) {
    if (!c || n < 0) return fail(c, GS_ERR_INVALID_ARG, "time must be >= 0");
    c->time = n;
    if (c->d_counter) {
        const long long v = n;
        GS_CUDA(c, cudaMemcpyAsync(c->d_counter, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return GS_OK;
}

gs_status gs_get_time(const gs_ctx* c, int64_t* out) {
    if (!c || !out) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context or output pointer");
    *out = c->time;
    return GS_OK;
}

gs_status gs_step(gs_ctx* c, int64_t n_iters, int64_t batch_size) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    if (n_iters < 0 || batch_size < 0) return fail(c, GS_ERR_INVALID_ARG, "n_iters and batch_size must be >= 0");
    gs_status st = ensure_descs(c);
    if (st != GS_OK) return st;
    if (n_iters == 0) return GS_OK;
    if (batch_size == 0) {
        // Listing 1: one launch per iteration (per fused group of depth t).
        cudaError_t err = cudaSuccess;
        int64_t launched = 0;
        for_each_launch(c, n_iters, c->parity, [&](LaunchDesc& d) {
            if (err == cudaSuccess) {
                err = launch_one(c, d);
                ++launched;
            }
        });
        c->stats.kernel_launches += launched;
        if (err != cudaSuccess) return cuda_fail(c, err, "kernel launch");
        c->parity ^= flip_of(c, n_iters);
    } else {
        // Listing 3 plus loop peeling: floor(n/S) graph launches of S
        // iterations, then one remainder graph of n mod S iterations.
        const int64_t nb = n_iters / batch_size;
        const int64_t r = n_iters - nb * batch_size;
        if (r > 0 && c->rem_S != r) {
            drop_remainder(c, batch_size);
            c->rem_S = r;
        }
        st = prepare_step_graphs(c, n_iters, batch_size);
        if (st != GS_OK) return st;
        if (nb > 0) {
            st = run_batches(c, batch_size, nb);
            if (st != GS_OK) return st;
        }
        if (r > 0) {
            st = launch_graphs(c, r, 1);
            if (st != GS_OK) return st;
        }
    }
    c->time += n_iters;
    c->stats.iterations += n_iters;
    return GS_OK;
}

gs_status gs_graph_build(gs_ctx* c, int64_t S) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    if (S < 1) return fail(c, GS_ERR_INVALID_ARG, "batch_size must be >= 1");
    gs_status st = ensure_descs(c);
    if (st != GS_OK) return st;
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    const int fl = flip_of(c, S);
    for (int p = 0; p < 2; ++p) {
        auto it = c->graphs.find(std::make_pair(S, p));
        if (it != c->graphs.end()) {
            cudaGraphExecDestroy(it->second.exec);
            cudaGraphDestroy(it->second.graph);
            c->graphs.erase(it);
        }
    }
    {
        auto it = c->loops.find(std::make_pair(S, c->parity));
        if (it != c->loops.end()) {
            cudaGraphExecDestroy(it->second.exec);
            cudaGraphDestroy(it->second.graph);
            c->loops.erase(it);
        }
    }
    const auto t0 = std::chrono::steady_clock::now();
    GraphEntry* e = nullptr;
    if (c->plan.graph_loop) {
        st = ensure_loop(c, S, c->parity, &e);
    } else {
        st = ensure_graph(c, S, c->parity, &e);
        if (st == GS_OK && fl) st = ensure_graph(c, S, c->parity ^ 1, &e);
    }
    if (st != GS_OK) return st;
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    const auto t1 = std::chrono::steady_clock::now();
    c->stats.last_build_seconds = std::chrono::duration<double>(t1 - t0).count();
    c->stats.last_build_nodes = e->nodes;
    c->built_S = S;
    return GS_OK;
}

gs_status gs_graph_launch(gs_ctx* c, int64_t n_launches) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    if (n_launches < 0) return fail(c, GS_ERR_INVALID_ARG, "n_launches must be >= 0");
    if (c->built_S == 0) return fail(c, GS_ERR_STATE, "no graph built (call gs_graph_build first)");
    gs_status st = run_batches(c, c->built_S, n_launches);
    if (st != GS_OK) return st;
    c->time += c->built_S * n_launches;
    c->stats.iterations += c->built_S * n_launches;
    return GS_OK;
}

gs_status gs_graph_destroy(gs_ctx* c) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    if (c->stream) cudaStreamSynchronize(c->stream);
    destroy_graphs(c);
    return GS_OK;
}

gs_status gs_sync(gs_ctx* c) {
    if (!c) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context");
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    GS_CUDA(c, cudaGetLastError());
    return GS_OK;
}

gs_status gs_get_stats(const gs_ctx* c, gs_stats* out) {
    if (!c || !out) return fail(nullptr, GS_ERR_INVALID_ARG, "NULL context or output pointer");
    *out = c->stats;
    return GS_OK;
}

}  // extern "C"
