// gs_multi_step_noalloc: the fused multi-instance step for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory all comes
// from its own allocator or a fixed budget (a host framework that forbids raw
// allocations outside its memory manager), and latency-critical loops that
// cannot afford cudaMalloc's implicit device synchronisation.  gs_multi_*
// allocates a descriptor table per batch; this entry point instead keeps the
// table in a fixed array in device memory that is part of the loaded library
// (every GPU that loads the library holds it until the process exits), so a
// call allocates nothing: the caller passes the fields (inputs and outputs)
// and the step runs the same persistent kernel as GS_MULTI_FUSED, one launch
// per iteration.
//
// The rows reach the table through the parameters of a small fill kernel
// (at most 64 rows a launch), not through a copy from host memory: kernel
// parameters are copied when the launch is issued, so nothing refers to the
// caller's stack once the call has returned.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include <cuda.h>

#include "common.cuh"

using namespace gs;

namespace {

// The shared descriptor table.  In host code this name is only a host-side
// stand-in for the device array: a kernel must be given the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) MultiInstance g_noalloc_desc[GS_NOALLOC_MAX_INSTANCES];

constexpr int kMaxDevices = 64;
constexpr int kBlockX = 64;     // threads per block (16-byte vectors along x)
constexpr int kRows = 8;        // rows per work item
constexpr int kFillRows = 64;   // table rows per fill launch (parameters < 4 KiB)

struct FillArgs {
    MultiInstance* dst;  // first table row to write
    int count;           // rows in this launch
    MultiInstance rows[kFillRows];
};
static_assert(sizeof(FillArgs) <= 4096, "fill parameters must fit the classic 4 KiB parameter space");

__global__ void noalloc_fill_kernel(const FillArgs a) {
    const int r = threadIdx.x;
    if (r < a.count) a.dst[r] = a.rows[r];
}

// Per device: the table's address and launch facts, resolved once for the
// CUDA context that was current when they were taken (keyed by that
// context's unique id, so a context created after cudaDeviceReset gets its
// own set-up instead of a stale address).
struct DeviceSetup {
    unsigned long long ctx_id = 0;  // 0: not set up
    MultiInstance* desc = nullptr;  // device address of g_noalloc_desc
    int sms = 0;
    int occ[3][2] = {};             // resident blocks per SM of the step kernel, [dtype][bc]
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

using PfnCtxGetCurrent = CUresult(CUDAAPI*)(CUcontext*);
using PfnCtxGetId = CUresult(CUDAAPI*)(CUcontext, unsigned long long*);

// The driver's cuCtxGetCurrent / cuCtxGetId, looked up once through the
// runtime (the library links no driver library).
struct DriverFns {
    PfnCtxGetCurrent get_current = nullptr;
    PfnCtxGetId get_id = nullptr;
    bool ok = false;
};
const DriverFns& driver_fns() {
    static const DriverFns fns = [] {
        DriverFns f;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f.get_current = reinterpret_cast<PfnCtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f.get_id = reinterpret_cast<PfnCtxGetId>(p);
        f.ok = f.get_current && f.get_id;
        return f;
    }();
    return fns;
}

// Unique id of the CUDA context current on this thread (0: none current).
cudaError_t current_ctx_id(unsigned long long* id) {
    *id = 0;
    const DriverFns& d = driver_fns();
    if (!d.ok) return cudaErrorNotSupported;
    CUcontext c = nullptr;
    if (d.get_current(&c) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    if (!c) return cudaSuccess;
    return d.get_id(c, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorContextIsDestroyed;
}

// With device `dev` current: the cached set-up if it belongs to the current
// context, else resolve the table's device address (cudaGetSymbolAddress,
// which also makes the device's primary context current on this thread),
// the SM count and the step kernels' occupancy, and cache them.
cudaError_t setup_device(int dev, DeviceSetup* out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    unsigned long long id = 0;
    cudaError_t e = current_ctx_id(&id);
    if (e != cudaSuccess) return e;
    if (id != 0 && id == s.ctx_id) {
        *out = s;
        return cudaSuccess;
    }
    DeviceSetup n;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_desc);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&n.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const gs_dtype dts[3] = {GS_F32, GS_BF16, GS_F16};
    const gs_bc bcs[2] = {GS_BC_CLAMP, GS_BC_DIRICHLET0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2; ++j) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n.occ[i][j], heat_multi_func(dts[i], bcs[j], GS_KERNEL_MARCH),
                                                              kBlockX, 0);
            if (e != cudaSuccess) return e;
        }
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, noalloc_fill_kernel);  // loads the fill kernel now, not on the first call
    if (e != cudaSuccess) return e;
    e = current_ctx_id(&n.ctx_id);
    if (e != cudaSuccess) return e;
    n.desc = static_cast<MultiInstance*>(p);
    s = n;
    *out = s;
    return cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// One buffer's byte range, for the overlap check.
struct Span {
    uintptr_t lo, hi;
    bool written;  // T0 / T1 (P is only read)
    int inst;
};

}  // namespace

extern "C" gs_status gs_multi_step_noalloc(const gs_instance* inst, int32_t n_inst, int32_t parity, int64_t n_iters,
                                           const gs_heat_coeffs* coeffs, gs_dtype storage, gs_bc bc, void* stream,
                                           int32_t* parity_out) {
    if (!inst || !coeffs) return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: NULL argument");
    if (n_inst < 1 || n_inst > GS_NOALLOC_MAX_INSTANCES)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: n_inst = " + std::to_string(n_inst) +
                                                   " outside [1, " + std::to_string(GS_NOALLOC_MAX_INSTANCES) +
                                                   "] (the fixed descriptor table's size)");
    if ((parity != 0 && parity != 1) || n_iters < 0)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: parity must be 0/1 and n_iters >= 0");
    if (storage != GS_F32 && storage != GS_BF16 && storage != GS_F16)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: unknown storage dtype");
    if (bc != GS_BC_CLAMP && bc != GS_BC_DIRICHLET0)
        return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: bc must be clamp or Dirichlet-0");
    const float cv[6] = {coeffs->k, coeffs->cx, coeffs->cy, coeffs->cz, coeffs->cz2, coeffs->t_amb};
    for (float v : cv)
        if (!std::isfinite(v)) return global_fail(GS_ERR_NUMERIC, "gs_multi_step_noalloc: non-finite coefficient");
    const int V = (storage == GS_F32) ? 4 : 8;
    const size_t eb = (storage == GS_F32) ? 4 : 2;
    const int span = kBlockX * V;

    // Descriptor rows on the stack, largest instances first.
    int order[GS_NOALLOC_MAX_INSTANCES];
    Span spans[3 * GS_NOALLOC_MAX_INSTANCES];
    for (int i = 0; i < n_inst; ++i) {
        const gs_instance& d = inst[i];
        const char* bad = nullptr;  // messages are built only on failure
        if (!d.T0 || !d.T1 || !d.P || !aligned16(d.T0) || !aligned16(d.T1) || !aligned16(d.P))
            bad = "T0, T1, P must be non-NULL and 16-byte aligned";
        else if (d.nx < 1 || d.ny < 1 || d.nx > (1 << 20) || d.ny > (1 << 20))
            bad = "nx, ny must be in [1, 2^20]";
        else if (d.pitch < d.nx || d.pitch % V || d.p_pitch < d.nx || d.p_pitch % V)
            bad = "pitches must be >= nx and a multiple of 16 bytes";
        if (bad)
            return global_fail(GS_ERR_INVALID_ARG,
                               "gs_multi_step_noalloc: instance " + std::to_string(i) + ": " + bad);
        order[i] = i;
        const uintptr_t tb = (uintptr_t)(d.pitch * d.ny) * eb, pb = (uintptr_t)(d.p_pitch * d.ny) * eb;
        spans[3 * i + 0] = Span{(uintptr_t)d.T0, (uintptr_t)d.T0 + tb, true, i};
        spans[3 * i + 1] = Span{(uintptr_t)d.T1, (uintptr_t)d.T1 + tb, true, i};
        spans[3 * i + 2] = Span{(uintptr_t)d.P, (uintptr_t)d.P + pb, false, i};
    }
    // No two buffers may overlap, except P buffers with each other (they are
    // only read): a written buffer that overlaps another buffer would be
    // updated while it is read.  Sorted by start, a buffer overlaps an
    // earlier one exactly when an earlier one ends past its start.
    {
        const int ns = 3 * n_inst;
        std::sort(spans, spans + ns, [](const Span& a, const Span& b) { return a.lo < b.lo; });
        uintptr_t end_any = 0, end_written = 0;
        int inst_any = -1, inst_written = -1;
        for (int k = 0; k < ns; ++k) {
            const Span& s = spans[k];
            const bool hit = s.written ? (end_any > s.lo) : (end_written > s.lo);
            if (hit) {
                const int other = s.written ? inst_any : inst_written;
                const std::string who = (other == s.inst) ? "instance " + std::to_string(s.inst) + ": its buffers"
                                                          : "buffers of instances " +
                                                                std::to_string(std::min(other, s.inst)) + " and " +
                                                                std::to_string(std::max(other, s.inst));
                return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: " + who +
                                                           " overlap (T0 and T1 of every instance need memory of "
                                                           "their own; only P buffers may be shared)");
            }
            if (s.hi > end_any) { end_any = s.hi; inst_any = s.inst; }
            if (s.written && s.hi > end_written) { end_written = s.hi; inst_written = s.inst; }
        }
    }
    std::stable_sort(order, order + n_inst,
                     [&](int a, int b) { return inst[a].nx * inst[a].ny > inst[b].nx * inst[b].ny; });
    FillArgs fill[(GS_NOALLOC_MAX_INSTANCES + kFillRows - 1) / kFillRows];
    int64_t items = 0;
    for (int k = 0; k < n_inst; ++k) {
        const gs_instance& d = inst[order[k]];
        MultiInstance& r = fill[k / kFillRows].rows[k % kFillRows];
        r.T0 = d.T0;
        r.T1 = d.T1;
        r.P = d.P;
        r.pitch = d.pitch;
        r.p_pitch = d.p_pitch;
        r.nx = (int)d.nx;
        r.ny = (int)d.ny;
        r.first_item = (int)items;
        r.n_items = (int)(((d.nx + span - 1) / span) * ((d.ny + kRows - 1) / kRows));
        items += r.n_items;
        if (items >= (int64_t(1) << 31))
            return global_fail(GS_ERR_INVALID_ARG, "gs_multi_step_noalloc: more than 2^31 work items");
    }
    if (parity_out) *parity_out = parity;
    if (n_iters == 0) return GS_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return global_fail(GS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return global_fail(GS_ERR_UNSUPPORTED, "device ordinal >= 64");
    DeviceSetup ds;
    e = setup_device(dev, &ds);
    if (e != cudaSuccess)
        return global_fail(GS_ERR_CUDA, std::string("gs_multi_step_noalloc set-up (table address, occupancy): ") +
                                            cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Overwrite the shared table (stream-ordered after earlier work on st).
    const int n_fill = (n_inst + kFillRows - 1) / kFillRows;
    for (int b = 0; b < n_fill; ++b) {
        FillArgs& f = fill[b];
        f.dst = ds.desc + b * kFillRows;
        f.count = std::min(kFillRows, n_inst - b * kFillRows);
        void* args[1] = {&f};
        e = cudaLaunchKernel((const void*)noalloc_fill_kernel, dim3(1), dim3(kFillRows), args, 0, st);
        if (e != cudaSuccess)
            return global_fail(GS_ERR_CUDA, std::string("descriptor table fill: ") + cudaGetErrorString(e));
    }

    const int di = (storage == GS_F32) ? 0 : (storage == GS_BF16 ? 1 : 2);
    const int occ = ds.occ[di][bc == GS_BC_CLAMP ? 0 : 1];
    const void* f = heat_multi_func(storage, bc, GS_KERNEL_MARCH);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)std::max(1, occ) * ds.sms));
    MultiArgs a{};
    a.desc = ds.desc;
    a.n_inst = n_inst;
    a.total_items = (int)items;
    a.rows = kRows;
    a.c = HeatCoef{coeffs->k, coeffs->cx, coeffs->cy, coeffs->cz, coeffs->cz2, coeffs->t_amb};
    int p = parity;
    for (int64_t it = 0; it < n_iters; ++it) {
        a.parity = p;
        void* args[1] = {&a};
        e = cudaLaunchKernel(f, dim3(blocks), dim3(kBlockX), args, 0, st);
        if (e != cudaSuccess) return global_fail(GS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        p ^= 1;
    }
    if (parity_out) *parity_out = p;
    return GS_OK;
}
