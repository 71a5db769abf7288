// The paper's skeleton application (Sec. III-C): a vector multiplied in
// place by a constant, one kernel launch per iteration.  Every graph node
// takes the same parameter block, as in the paper's Listing 3.
#include <algorithm>

#include "common.cuh"

namespace gs {

template <typename ST>
__global__ void __launch_bounds__(256) skeleton_kernel(const SkeletonArgs a) {
    constexpr int V = Vec<ST>::N;
    pdl_wait_then_trigger();
    ST* x = static_cast<ST*>(a.x);
    const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (i0 >= a.n) return;
    float v[V];
    load_vec_rw(x + i0, v);
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = __fmul_rn(a.c, v[e]);
    store_vec(x + i0, v, (a.n - i0 < V) ? (int)(a.n - i0) : V);
}

cudaError_t skeleton_desc(gs_dtype dt, const SkeletonArgs& a, int block_x, LaunchDesc* out) {
    const int V = (dt == GS_F32) ? 4 : 8;
    switch (dt) {
        case GS_F32: out->func = (const void*)skeleton_kernel<float>; break;
        case GS_BF16: out->func = (const void*)skeleton_kernel<__nv_bfloat16>; break;
        case GS_F16: out->func = (const void*)skeleton_kernel<__half>; break;
        default: return cudaErrorInvalidValue;
    }
    const long long vecs = (a.n + V - 1) / V;
    out->block = dim3(block_x, 1, 1);
    out->grid = dim3((unsigned)std::max<long long>(1, (vecs + block_x - 1) / block_x), 1, 1);
    out->smem = 0;
    out->set_args(a);
    return cudaSuccess;
}

}  // namespace gs
