// Internal declarations shared by the library's translation units (not part
// of the public C ABI; see include/graphstep.h for that).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "graphstep.h"

namespace gs {

// ---------------------------------------------------------------- storage --
// Fields are stored as f32, bf16 or f16; every kernel loads 16-byte vectors,
// widens to f32, computes in f32 and rounds to nearest even on store.

template <typename ST> struct Vec;  // elements per 16-byte vector

template <> struct Vec<float> { static constexpr int N = 4; };
template <> struct Vec<__nv_bfloat16> { static constexpr int N = 8; };
template <> struct Vec<__half> { static constexpr int N = 8; };

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

template <typename ST> __device__ __forceinline__ ST from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// ------------------------------------------------------- checked build --
// With GS_CHECKED defined, the translation units that also define
// GS_CHECK_THIS_UNIT (the stencil kernels) check every global field access
// of the helpers below against a table of registered byte ranges (set from
// the host, gs_debug_check_ranges): an access outside every range is
// counted, its address recorded, and skipped (a load gives zeros).  Nothing
// faults.  Each translation unit has its own table (no relocatable device
// code), filled through its <unit>_check_set / _check_get functions.
constexpr int kCheckRanges = 128;
#if defined(GS_CHECKED) && defined(GS_CHECK_THIS_UNIT)
static __device__ unsigned long long g_chk_lo[kCheckRanges], g_chk_hi[kCheckRanges];
static __device__ int g_chk_n;
static __device__ unsigned long long g_chk_bad, g_chk_first;
__device__ __forceinline__ bool gs_chk(const void* p, size_t bytes) {
    const unsigned long long lo = reinterpret_cast<unsigned long long>(p), hi = lo + bytes;
    const int n = g_chk_n;
    for (int i = 0; i < n; ++i)
        if (lo >= g_chk_lo[i] && hi <= g_chk_hi[i]) return true;
    if (atomicAdd(&g_chk_bad, 1ull) == 0ull) g_chk_first = lo;
    return false;
}
#define GS_CHK(p, bytes) gs_chk((p), (bytes))
#define GS_CHECK_UNIT(NAME)                                                                                  \
    cudaError_t NAME##_check_set(const unsigned long long* lo, const unsigned long long* hi, int n) {         \
        cudaError_t e = cudaMemcpyToSymbol(g_chk_lo, lo, sizeof(unsigned long long) * n);                     \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_chk_hi, hi, sizeof(unsigned long long) * n);           \
        const unsigned long long zero = 0;                                                                    \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_chk_n, &n, sizeof(int));                               \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_chk_bad, &zero, sizeof(zero));                          \
        return e;                                                                                             \
    }                                                                                                         \
    cudaError_t NAME##_check_get(unsigned long long* bad, unsigned long long* first) {                         \
        cudaError_t e = cudaMemcpyFromSymbol(bad, g_chk_bad, sizeof(*bad));                                   \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(first, g_chk_first, sizeof(*first));                   \
        const unsigned long long zero = 0;                                                                    \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_chk_bad, &zero, sizeof(zero));                          \
        return e;                                                                                             \
    }
#else
#define GS_CHK(p, bytes) true
#define GS_CHECK_UNIT(NAME)                                                                                  \
    cudaError_t NAME##_check_set(const unsigned long long*, const unsigned long long*, int) {                 \
        return cudaErrorNotSupported;                                                                         \
    }                                                                                                         \
    cudaError_t NAME##_check_get(unsigned long long*, unsigned long long*) { return cudaErrorNotSupported; }
#endif
cudaError_t heat_check_set(const unsigned long long* lo, const unsigned long long* hi, int n);
cudaError_t heat_check_get(unsigned long long* bad, unsigned long long* first);
cudaError_t fdtd_check_set(const unsigned long long* lo, const unsigned long long* hi, int n);
cudaError_t fdtd_check_get(unsigned long long* bad, unsigned long long* first);

// 16-byte vector load through the read-only path.
template <typename ST>
__device__ __forceinline__ void load_vec(const ST* __restrict__ p, float (&v)[Vec<ST>::N]) {
    if (!GS_CHK(p, 16)) {
#pragma unroll
        for (int i = 0; i < Vec<ST>::N; ++i) v[i] = 0.f;
        return;
    }
    const uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
    const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
    for (int i = 0; i < Vec<ST>::N; ++i) v[i] = to_f32(e[i]);
}

// 16-byte vector load through the coherent path (for in-place updates).
template <typename ST>
__device__ __forceinline__ void load_vec_rw(const ST* p, float (&v)[Vec<ST>::N]) {
    if (!GS_CHK(p, 16)) {
#pragma unroll
        for (int i = 0; i < Vec<ST>::N; ++i) v[i] = 0.f;
        return;
    }
    const uint4 raw = *reinterpret_cast<const uint4*>(p);
    const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
    for (int i = 0; i < Vec<ST>::N; ++i) v[i] = to_f32(e[i]);
}

// Store a vector; `n_valid` < N stores only the first n_valid elements.
template <typename ST>
__device__ __forceinline__ void store_vec(ST* p, const float (&v)[Vec<ST>::N], int n_valid) {
    constexpr int N = Vec<ST>::N;
    if (!GS_CHK(p, sizeof(ST) * (n_valid >= N ? N : (n_valid > 0 ? n_valid : 0)))) return;
    if (n_valid >= N) {
        uint4 raw;
        ST* e = reinterpret_cast<ST*>(&raw);
#pragma unroll
        for (int i = 0; i < N; ++i) e[i] = from_f32<ST>(v[i]);
        *reinterpret_cast<uint4*>(p) = raw;
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < n_valid) p[i] = from_f32<ST>(v[i]);
    }
}

template <typename ST>
__device__ __forceinline__ float load_scalar(const ST* p) { return GS_CHK(p, sizeof(ST)) ? to_f32(__ldg(p)) : 0.f; }

// One element through the coherent path (a value the launch may write).
template <typename ST>
__device__ __forceinline__ float load_scalar_rw(const ST* p) { return GS_CHK(p, sizeof(ST)) ? to_f32(*p) : 0.f; }

template <typename ST>
__device__ __forceinline__ void store_scalar(ST* p, float v) {
    if (GS_CHK(p, sizeof(ST))) *p = from_f32<ST>(v);
}

// One uint8 material id.
__device__ __forceinline__ unsigned load_id(const unsigned char* p) { return GS_CHK(p, 1) ? __ldg(p) : 0u; }

// W elements per access, W * sizeof(ST) = 4, 8 or 16 bytes (read-only path).
template <typename ST, int W>
__device__ __forceinline__ void load_vecw(const ST* __restrict__ p, float (&v)[W]) {
    static_assert(W * sizeof(ST) == 4 || W * sizeof(ST) == 8 || W * sizeof(ST) == 16, "4-, 8- or 16-byte access");
    if (!GS_CHK(p, W * sizeof(ST))) {
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = 0.f;
        return;
    }
    if constexpr (W * sizeof(ST) == 16) {
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(p));
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    } else if constexpr (W * sizeof(ST) == 4) {
        const unsigned raw = __ldg(reinterpret_cast<const unsigned*>(p));
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    } else {
        const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    }
}

// W elements per access through the coherent path (for in-place updates).
template <typename ST, int W>
__device__ __forceinline__ void load_vecw_rw(const ST* p, float (&v)[W]) {
    static_assert(W * sizeof(ST) == 8 || W * sizeof(ST) == 16, "8- or 16-byte access");
    if (!GS_CHK(p, W * sizeof(ST))) {
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = 0.f;
        return;
    }
    if constexpr (W * sizeof(ST) == 16) {
        const uint4 raw = *reinterpret_cast<const uint4*>(p);
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    } else {
        const uint2 raw = *reinterpret_cast<const uint2*>(p);
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    }
}

// W consecutive uint8 ids (W = 4 or 8: a 4- or 8-byte access).
template <int W>
__device__ __forceinline__ void load_ids(const unsigned char* __restrict__ p, unsigned (&id)[W]) {
    static_assert(W == 4 || W == 8, "4 or 8 ids");
    if (!GS_CHK(p, W)) {
#pragma unroll
        for (int i = 0; i < W; ++i) id[i] = 0u;
        return;
    }
    if constexpr (W == 4) {
        const unsigned raw = __ldg(reinterpret_cast<const unsigned*>(p));
#pragma unroll
        for (int i = 0; i < 4; ++i) id[i] = (raw >> (8 * i)) & 0xffu;
    } else {
        const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            id[i] = (raw.x >> (8 * i)) & 0xffu;
            id[4 + i] = (raw.y >> (8 * i)) & 0xffu;
        }
    }
}

template <typename ST, int W>
__device__ __forceinline__ void store_vecw(ST* p, const float (&v)[W], int n_valid) {
    if (!GS_CHK(p, sizeof(ST) * (n_valid >= W ? W : (n_valid > 0 ? n_valid : 0)))) return;
    if (n_valid >= W) {
        if constexpr (W * sizeof(ST) == 16) {
            uint4 raw;
            ST* e = reinterpret_cast<ST*>(&raw);
#pragma unroll
            for (int i = 0; i < W; ++i) e[i] = from_f32<ST>(v[i]);
            *reinterpret_cast<uint4*>(p) = raw;
        } else if constexpr (W * sizeof(ST) == 4) {
            unsigned raw;
            ST* e = reinterpret_cast<ST*>(&raw);
#pragma unroll
            for (int i = 0; i < W; ++i) e[i] = from_f32<ST>(v[i]);
            *reinterpret_cast<unsigned*>(p) = raw;
        } else {
            uint2 raw;
            ST* e = reinterpret_cast<ST*>(&raw);
#pragma unroll
            for (int i = 0; i < W; ++i) e[i] = from_f32<ST>(v[i]);
            *reinterpret_cast<uint2*>(p) = raw;
        }
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i)
            if (i < n_valid) p[i] = from_f32<ST>(v[i]);
    }
}

// Programmatic dependent launch: a kernel first waits until the grid it
// depends on has completed and its memory is visible, then lets its own
// dependent start launching.  Waiting first keeps the early launch to one
// kernel ahead (triggering first would let the whole chain launch at once
// and fill the SMs with waiting blocks).  Both are no-ops when the launch
// had no programmatic dependency.
__device__ __forceinline__ void pdl_wait_then_trigger() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The launch's block index, walked last to first when `rev` is set: with
// consecutive launches alternating, a step starts on the blocks the previous
// step ran last, whose rows are still in L2 (gs_traverse).
__device__ __forceinline__ uint3 block_index(int rev) {
    if (!rev) return blockIdx;
    return make_uint3(gridDim.x - 1 - blockIdx.x, gridDim.y - 1 - blockIdx.y, gridDim.z - 1 - blockIdx.z);
}

// ---------------------------------------------------------- kernel args --

struct HeatCoef {
    float k, cx, cy, cz, cz2, t_amb;
};

struct HeatArgs {
    const void* Tin;
    void* Tout;
    const void* P;
    int nx, ny, nz;
    int rows;            // y rows per block (depth-1 kernels)
    long long pitch;     // elements per row
    long long plane;     // elements per z plane (pitch * ny)
    long long p_pitch;   // elements per row of P
    int tile_x, tile_y;  // output tile (temporal kernels)
    int rev;             // walk the blocks last to first (block_index)
    HeatCoef c;
};

struct FdtdArgs {
    void* f[6];           // Ex, Ey, Ez, Hx, Hy, Hz
    void* g[6];           // fused step: the set written (f is read); unused otherwise
    int N;                // cells along i and j
    int Nk;               // cells along k (N for a cube; a sub-domain of a slab set may differ)
    int kc;               // k planes per block
    int kmarch;           // fused step: k planes a block marches (0: one plane a thread, no march)
    long long pitch;      // elements per row (>= N+1)
    long long plane;      // pitch * (N+1)
    float s;              // courant number
    int src_on;
    int si, sj, sk;
    float amp, delay, width;
    long long* counter;   // device step counter (E kernel, source owner)
    // Media (NULL mat: vacuum): uint8 material ids at the components' own
    // element offsets, and the coefficient table: med[m] = (da, db) of the
    // H update, med[256 + m] = (ca, cb) of the E update, for all 256 ids.
    const unsigned char* mat;
    const float2* med;
    int rev;              // walk the blocks last to first (block_index)
};

struct SkeletonArgs {
    void* x;
    long long n;
    float c;
};

// One instance of the persistent multi-instance kernel (device table row).
struct MultiInstance {
    void* T0;
    void* T1;
    const void* P;
    long long pitch, p_pitch;
    int nx, ny;
    int first_item;  // index of this instance's first (x tile, y tile) item
    int n_items;
};

struct MultiArgs {
    const MultiInstance* desc;  // device table, n_inst rows, largest first
    int n_inst;
    int total_items;
    int rows;
    int parity;  // 0: read T0, write T1; 1: the reverse
    int rev;     // take the work items last to first
    HeatCoef c;
};

// A ready-to-launch kernel: host stub, launch shape and its single by-value
// argument (every kernel here takes exactly one struct argument).
struct LaunchDesc {
    const void* func = nullptr;
    dim3 grid, block;
    size_t smem = 0;
    alignas(16) unsigned char args[256];
    size_t args_size = 0;

    template <typename A> void set_args(const A& a) {
        static_assert(sizeof(A) <= sizeof(args), "kernel args too large");
        memcpy(args, &a, sizeof(A));
        args_size = sizeof(A);
    }
    void* arg_ptr() { return args; }
};

// Kernel factories implemented in heat.cu / fdtd.cu / convert.cu.  They
// return cudaSuccess or the first CUDA error (e.g. from setting the dynamic
// shared memory limit), and cudaErrorInvalidValue for unsupported shapes.
// Thermal kernel variants (gs_plan.kernel).
constexpr int kWaveMaxNz = 16;   // wavefront kernel holds all planes in one block
constexpr int kColumnMaxNz = 8;  // column kernel holds all planes in registers
cudaError_t heat_desc(gs_kind kind, gs_dtype dt, gs_bc bc, const HeatArgs& a, int block_x, int depth, int variant,
                      LaunchDesc* out);
size_t heat_temporal_smem(int nz, int tile_x, int tile_y, int depth);
size_t heat_wave_smem(int nz3d, int depth, int vec);
size_t heat_scol_smem(int nzm, int rows, int vec);
// STREAM kernel (3D, depth 2): dynamic shared memory of a block (block_x 512:
// 16 compute warps, else 8), and the count of its bounded stage waits that
// ran out since the last call (read and cleared; ~0u if the read failed).
size_t heat_stream_smem(gs_dtype dt, int block_x);
unsigned heat_stream_timeouts_take();
// heat_multi_kernel for (dt, bc) with MARCH tiles (blockDim.x threads x
// `rows` rows) or COLUMN tiles (32 x `rows` threads, one row per warp row),
// the latter also at temporal depth 2 or 4 (NULL for other combinations).
const void* heat_multi_func(gs_dtype dt, gs_bc bc, int variant, int depth = 1);
// Cells along x and rows along y of one work item of that kernel.
int heat_multi_span(gs_dtype dt, int variant, int depth, int block_x);
int heat_multi_item_rows(gs_dtype dt, int variant, int depth, int rows);
// FDTD H (e_half false) or E kernel; variant GS_KERNEL_COLUMN (no march,
// block (32, kc, 8/kc)) or GS_KERNEL_MARCH (block_x threads marching kc planes).
cudaError_t fdtd_desc(gs_dtype dt, bool e_half, const FdtdArgs& a, int block_x, int variant, LaunchDesc* out);
cudaError_t convert_to_storage(gs_dtype dt, const float* src, void* dst, long long width, long long rows,
                               long long pitch, cudaStream_t st);
cudaError_t convert_from_storage(gs_dtype dt, const void* src, float* dst, long long width, long long rows,
                                 long long pitch, cudaStream_t st);

cudaError_t skeleton_desc(gs_dtype dt, const SkeletonArgs& a, int block_x, LaunchDesc* out);

// Host-side fault injection (gs_debug_inject_failure): every device
// allocation and graph kernel-node addition of the library goes through
// these, which fail the armed call once with cudaErrorMemoryAllocation /
// cudaErrorInvalidValue and otherwise forward to CUDA.
cudaError_t gs_malloc_raw(void** p, size_t bytes);
template <typename T> cudaError_t gs_malloc(T** p, size_t bytes) { return gs_malloc_raw(reinterpret_cast<void**>(p), bytes); }
cudaError_t gs_graph_add_kernel_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t n,
                                     const cudaKernelNodeParams* params);

int device_sm_count();
size_t device_l2_bytes();
// Whether consecutive launches alternate their block order (gs_traverse):
// `mode` as given, AUTO deciding on the bytes one step touches.
bool traverse_alternates(int mode, double step_bytes);

// Accessors of a context for the other translation units.
void ctx_field(const gs_ctx* c, int id, void** ptr, int64_t* pitch);  // NULL / 0 if unbound
bool ctx_shape(const gs_ctx* c, int id, int64_t* width, int64_t* rows);
size_t ctx_elem_bytes(const gs_ctx* c);
bool ctx_is_heat(const gs_ctx* c);
bool ctx_is_skel(const gs_ctx* c);
cudaStream_t ctx_stream(const gs_ctx* c);
gs_status ctx_fail(gs_ctx* c, gs_status s, const std::string& msg);  // records msg, returns s
// gs_create; fdtd_box also admits FDTD grids of N x N x nz cells (nz != N),
// the sub-domains of a slab set.
gs_status ctx_create(gs_ctx** out, gs_kind kind, int64_t nx, int64_t ny, int64_t nz, gs_dtype storage, gs_bc bc,
                     void* stream, bool fdtd_box);
// The context's launch descriptors, built if needed (GS_ERR_STATE for
// unbound fields).
gs_status ctx_prepare(gs_ctx* c);
// The launches of n iterations starting at buffer parity p, in order
// (thermal: n/t depth-t launches, then n mod t depth-1 launches; FDTD: H, E
// per iteration); valid until the context's plan, fields or coefficients change.
void ctx_launch_list(gs_ctx* c, int64_t n, int p, std::vector<LaunchDesc*>* out);
// Buffer-parity flip of n iterations (thermal), 0 otherwise.
int ctx_flip(const gs_ctx* c, int64_t n);
// The context's kind, storage type and grid (n_iters: its step count).
void ctx_workload(const gs_ctx* c, gs_workload* w);
// One launch on the context's stream (with the plan's PDL attribute).
cudaError_t ctx_launch(gs_ctx* c, LaunchDesc& d);
gs_status global_fail(gs_status s, const std::string& msg);  // message for gs_last_error(NULL)

}  // namespace gs
