// Conversions between a dense float32 staging array (x fastest, no padding)
// and a pitched field in its storage type.  Used by gs_upload /
// gs_read_field for bf16 and f16 fields (f32 fields are copied directly).
// Rounding to storage is round-to-nearest-even.
#include "common.cuh"

namespace gs {

template <typename ST>
__global__ void to_storage_kernel(const float* __restrict__ src, ST* __restrict__ dst, long long width,
                                  long long rows, long long pitch) {
    const long long n = width * rows;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / width, x = idx - r * width;
        dst[r * pitch + x] = from_f32<ST>(src[idx]);
    }
}

template <typename ST>
__global__ void from_storage_kernel(const ST* __restrict__ src, float* __restrict__ dst, long long width,
                                    long long rows, long long pitch) {
    const long long n = width * rows;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / width, x = idx - r * width;
        dst[idx] = to_f32(src[r * pitch + x]);
    }
}

static unsigned grid_for(long long n) {
    const long long cap = (long long)device_sm_count() * 8;
    long long g = (n + 255) / 256;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

cudaError_t convert_to_storage(gs_dtype dt, const float* src, void* dst, long long width, long long rows,
                               long long pitch, cudaStream_t st) {
    const unsigned g = grid_for(width * rows);
    switch (dt) {
        case GS_BF16:
            to_storage_kernel<<<g, 256, 0, st>>>(src, static_cast<__nv_bfloat16*>(dst), width, rows, pitch);
            break;
        case GS_F16: to_storage_kernel<<<g, 256, 0, st>>>(src, static_cast<__half*>(dst), width, rows, pitch); break;
        case GS_F32: to_storage_kernel<<<g, 256, 0, st>>>(src, static_cast<float*>(dst), width, rows, pitch); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t convert_from_storage(gs_dtype dt, const void* src, float* dst, long long width, long long rows,
                                 long long pitch, cudaStream_t st) {
    const unsigned g = grid_for(width * rows);
    switch (dt) {
        case GS_BF16:
            from_storage_kernel<<<g, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(src), dst, width, rows, pitch);
            break;
        case GS_F16:
            from_storage_kernel<<<g, 256, 0, st>>>(static_cast<const __half*>(src), dst, width, rows, pitch);
            break;
        case GS_F32:
            from_storage_kernel<<<g, 256, 0, st>>>(static_cast<const float*>(src), dst, width, rows, pitch);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gs
