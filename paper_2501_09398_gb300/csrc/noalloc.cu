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
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"

using namespace gs;

namespace {

// The shared descriptor table.  In host code this name is only a host-side
// stand-in for the device array: a kernel must be given the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) MultiInstance g_noalloc_desc[GS_NOALLOC_MAX_INSTANCES];

constexpr int kMaxDevices = 64;
constexpr int kBlockX = 64;  // threads per block (16-byte vectors along x)
constexpr int kRows = 8;     // rows per work item

struct DeviceSetup {
    MultiInstance* desc = nullptr;  // device address of g_noalloc_desc
    int sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: resolve the table's device
// address and the SM count.
cudaError_t setup_device(int dev, DeviceSetup* out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.desc) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_desc);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        s.sms = sms;
        s.desc = static_cast<MultiInstance*>(p);
    }
    *out = s;
    return cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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
    const int span = kBlockX * V;

    // Descriptor rows on the stack, largest instances first.
    int order[GS_NOALLOC_MAX_INSTANCES];
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
    }
    std::stable_sort(order, order + n_inst,
                     [&](int a, int b) { return inst[a].nx * inst[a].ny > inst[b].nx * inst[b].ny; });
    MultiInstance rows[GS_NOALLOC_MAX_INSTANCES];
    int64_t items = 0;
    for (int k = 0; k < n_inst; ++k) {
        const gs_instance& d = inst[order[k]];
        MultiInstance& r = rows[k];
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
        return global_fail(GS_ERR_CUDA, std::string("cudaGetSymbolAddress of the descriptor table: ") +
                                            cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Overwrite the shared table (stream-ordered after earlier work on st;
    // the stack rows are staged by the runtime before the call returns).
    e = cudaMemcpyAsync(ds.desc, rows, sizeof(MultiInstance) * n_inst, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return global_fail(GS_ERR_CUDA, std::string("descriptor copy: ") + cudaGetErrorString(e));

    const void* f = heat_multi_func(storage, bc, GS_KERNEL_MARCH);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kBlockX, 0);
    if (e != cudaSuccess) return global_fail(GS_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
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
