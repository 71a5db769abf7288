// Learned cost model: an 18-32-32-1 ReLU MLP predicting log(ms per
// iteration) of a (workload, candidate) pair, trained and evaluated by the
// kernels in this file.  Parameters are one flat FP32 array:
//   W1[32][18] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3      (1697 floats)
// Inputs are standardised inside the kernels: xh = (x - mean) * inv_std.
// Loss: L = (1/N) sum_r (pred_r - y_r)^2 over the N rows of a batch.
// Training: Adam (beta1 0.9, beta2 0.999, eps 1e-8); one epoch of
// minibatches (fixed order) is built once as a graph of 2 nodes per
// minibatch and replayed per epoch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace {
#include "costmodel_weights.inc"
}  // namespace

namespace gs {
bool ctx_has_media(const gs_ctx* c);  // api.cu: an FDTD media table is set
}  // namespace gs

using namespace gs;

namespace {

constexpr int NI = GS_MLP_INPUTS;   // 18
constexpr int NH = GS_MLP_HIDDEN;   // 32
constexpr int NP = GS_MLP_PARAMS;   // 1697
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
static_assert(OB3 + 1 == NP, "parameter layout");
constexpr int ROWS = 128;           // rows per block (threads per block)
constexpr int PSTRIDE = NP + 1;     // per-block partial: NP gradients + loss

struct FwdBwdArgs {
    const float* params;
    const float* mean;
    const float* inv_std;
    const float* X;
    const float* y;
    long long row0, n_rows;  // rows [row0, row0 + n_rows) of X / y
    float scale;             // 2 / N
    float* partial;          // [gridDim.x][PSTRIDE]
    long long* step;         // Adam step counter, incremented once per launch (may be NULL)
};

struct ReduceAdamArgs {
    const float* partial;
    int n_blocks;
    float* grad;             // reduced gradient (NP) or NULL
    float* loss;             // reduced loss or NULL
    float* params;
    float* m;
    float* v;
    const long long* step;
    float lr;
    int update;              // 1: apply Adam
};

// One block = up to 128 rows.  Phase 1: each thread runs the forward and
// backward pass of one row, keeping only its 16 inputs in registers and
// writing activations and deltas to shared memory, feature-major with a
// padded stride (conflict-free in both phases).  Phase 2: the block's threads
// sum the weight gradients over its rows (fixed order) into this block's
// partial vector.
constexpr int RS = ROWS + 1;  // shared-memory stride of one feature's rows

__global__ void __launch_bounds__(ROWS) mlp_fwd_bwd_kernel(const FwdBwdArgs a) {
    extern __shared__ float sm[];
    float* P = sm;                      // NP
    float* xs = P + NP;                 // [NI][RS]
    float* h1s = xs + NI * RS;          // [NH][RS]
    float* h2s = h1s + NH * RS;         // [NH][RS]
    float* d1s = h2s + NH * RS;         // [NH][RS]
    float* d2s = d1s + NH * RS;         // [NH][RS]
    float* ds = d2s + NH * RS;          // [ROWS]
    float* ls = ds + ROWS;              // [ROWS] squared errors
    pdl_wait_then_trigger();
    const int t = threadIdx.x;
    for (int i = t; i < NP; i += ROWS) P[i] = a.params[i];
    if (a.step && blockIdx.x == 0 && t == 0) *a.step += 1;
    __syncthreads();

    const long long r = (long long)blockIdx.x * ROWS + t;  // row within the batch
    const bool valid = r < a.n_rows;
    float x[NI];
    float d = 0.f, se = 0.f;
    if (valid) {
        const float* xr = a.X + (a.row0 + r) * NI;
#pragma unroll
        for (int k = 0; k < NI; ++k) x[k] = (xr[k] - a.mean[k]) * a.inv_std[k];
    } else {
#pragma unroll
        for (int k = 0; k < NI; ++k) x[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < NI; ++k) xs[k * RS + t] = x[k];
    for (int i = 0; i < NH; ++i) {  // layer 1
        float acc = P[OB1 + i];
#pragma unroll
        for (int k = 0; k < NI; ++k) acc = fmaf(P[OW1 + i * NI + k], x[k], acc);
        h1s[i * RS + t] = valid ? fmaxf(acc, 0.f) : 0.f;
    }
    float pred = P[OB3];
    for (int i = 0; i < NH; ++i) {  // layer 2 and output
        float acc = P[OB2 + i];
#pragma unroll 8
        for (int j = 0; j < NH; ++j) acc = fmaf(P[OW2 + i * NH + j], h1s[j * RS + t], acc);
        const float h2 = valid ? fmaxf(acc, 0.f) : 0.f;
        h2s[i * RS + t] = h2;
        pred = fmaf(P[OW3 + i], h2, pred);
    }
    if (valid) {
        const float err = pred - a.y[a.row0 + r];
        se = err * err;
        d = a.scale * err;  // dL/dpred
    }
    for (int i = 0; i < NH; ++i)  // delta at layer-2 pre-activations
        d2s[i * RS + t] = (h2s[i * RS + t] > 0.f) ? d * P[OW3 + i] : 0.f;
    for (int j = 0; j < NH; ++j) {  // delta at layer-1 pre-activations
        float acc = 0.f;
#pragma unroll 8
        for (int i = 0; i < NH; ++i) acc = fmaf(P[OW2 + i * NH + j], d2s[i * RS + t], acc);
        d1s[j * RS + t] = (h1s[j * RS + t] > 0.f) ? acc : 0.f;
    }
    ds[t] = d;
    ls[t] = se;
    __syncthreads();

    float* out = a.partial + (size_t)blockIdx.x * PSTRIDE;
    for (int e = t; e < NP; e += ROWS) {
        float acc = 0.f;
        if (e < OB1) {                       // W1[i][k] = sum dh1[i] x[k]
            const int i = e / NI, k = e % NI;
            for (int q = 0; q < ROWS; ++q) acc = fmaf(d1s[i * RS + q], xs[k * RS + q], acc);
        } else if (e < OW2) {                // b1[i]
            const int i = e - OB1;
            for (int q = 0; q < ROWS; ++q) acc += d1s[i * RS + q];
        } else if (e < OB2) {                // W2[i][j] = sum dh2[i] h1[j]
            const int i = (e - OW2) / NH, j = (e - OW2) % NH;
            for (int q = 0; q < ROWS; ++q) acc = fmaf(d2s[i * RS + q], h1s[j * RS + q], acc);
        } else if (e < OW3) {                // b2[i]
            const int i = e - OB2;
            for (int q = 0; q < ROWS; ++q) acc += d2s[i * RS + q];
        } else if (e < OB3) {                // W3[j] = sum d h2[j]
            const int j = e - OW3;
            for (int q = 0; q < ROWS; ++q) acc = fmaf(ds[q], h2s[j * RS + q], acc);
        } else {                             // b3
            for (int q = 0; q < ROWS; ++q) acc += ds[q];
        }
        out[e] = acc;
    }
    if (t == 0) {
        float acc = 0.f;
        for (int q = 0; q < ROWS; ++q) acc += ls[q];
        out[NP] = acc;
    }
}

// Thread per parameter: sum the per-block partials in block order, then
// (optionally) one Adam update with bias correction for step *a.step.
__global__ void __launch_bounds__(256) mlp_reduce_adam_kernel(const ReduceAdamArgs a) {
    pdl_wait_then_trigger();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float g = 0.f;
    for (int b = 0; b < a.n_blocks; ++b) g += a.partial[(size_t)b * PSTRIDE + p];
    if (p == NP) {
        if (a.loss) *a.loss = g;
        return;
    }
    if (a.grad) a.grad[p] = g;
    if (a.update) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float t = (float)(*a.step);
        const float m = b1 * a.m[p] + (1.f - b1) * g;
        const float v = b2 * a.v[p] + (1.f - b2) * g * g;
        a.m[p] = m;
        a.v[p] = v;
        const float mh = m / (1.f - powf(b1, t));
        const float vh = v / (1.f - powf(b2, t));
        a.params[p] -= a.lr * mh / (sqrtf(vh) + eps);
    }
}

// ACC: add the prediction to out[r] (ensemble sums) instead of storing it.
template <bool ACC>
__global__ void __launch_bounds__(256) mlp_predict_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ mean,
                                                          const float* __restrict__ inv_std,
                                                          const float* __restrict__ X, long long n,
                                                          float* __restrict__ out) {
    __shared__ float P[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[NI], h1[NH];
#pragma unroll
    for (int k = 0; k < NI; ++k) x[k] = (X[r * NI + k] - mean[k]) * inv_std[k];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        float acc = P[OB1 + i];
#pragma unroll
        for (int k = 0; k < NI; ++k) acc = fmaf(P[OW1 + i * NI + k], x[k], acc);
        h1[i] = fmaxf(acc, 0.f);
    }
    float pred = P[OB3];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        float acc = P[OB2 + i];
#pragma unroll
        for (int j = 0; j < NH; ++j) acc = fmaf(P[OW2 + i * NH + j], h1[j], acc);
        pred = fmaf(P[OW3 + i], fmaxf(acc, 0.f), pred);
    }
    out[r] = ACC ? out[r] + pred : pred;
}

// Single block: index of the smallest value (ties: smallest index).
__global__ void __launch_bounds__(1024) argmin_kernel(const float* __restrict__ v, long long n,
                                                      long long* __restrict__ idx_out, float* __restrict__ val_out) {
    __shared__ float bv[1024];
    __shared__ long long bi[1024];
    float best = INFINITY;
    long long bidx = -1;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float x = v[i];
        if (x < best) { best = x; bidx = i; }  // ascending i: first minimum kept
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const float o = bv[threadIdx.x + s];
            const long long oi = bi[threadIdx.x + s];
            if (oi >= 0 && (bi[threadIdx.x] < 0 || o < bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x]))) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *idx_out = bi[0];
        *val_out = bv[0];
    }
}

// One block per feature: mean and 1/std (population), two passes in FP32.
__global__ void __launch_bounds__(256) norm_kernel(const float* __restrict__ X, long long n, float* mean,
                                                   float* inv_std) {
    __shared__ float red[256];
    const int k = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) s += X[r * NI + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const float mu = red[0] / (float)n;
    __syncthreads();
    float q = 0.f;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) {
        const float dv = X[r * NI + k] - mu;
        q += dv * dv;
    }
    red[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float sd = sqrtf(red[0] / (float)n);
        mean[k] = mu;
        inv_std[k] = (sd > 1e-6f) ? 1.f / sd : 1.f;  // constant features pass through centred
    }
}

constexpr size_t kFwdBwdSmem = (size_t)(NP + NI * RS + 4 * NH * RS + 2 * ROWS) * sizeof(float);

// splitmix64 (Steele, Lea, Flood 2014): deterministic weight initialisation.
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct gs_mlp {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float* params = nullptr;   // NP
    float* m = nullptr;        // NP
    float* v = nullptr;        // NP
    float* grad = nullptr;     // NP
    float* norm = nullptr;     // mean[NI] | inv_std[NI]
    float* loss = nullptr;     // 1
    long long* step = nullptr; // Adam step counter
    float* partial = nullptr;  // [cap_blocks][PSTRIDE]
    int cap_blocks = 0;
    float* pred = nullptr;     // prediction scratch for argmin
    long long pred_cap = 0;
    long long* amin_idx = nullptr;
    float* amin_val = nullptr;
    std::string err;
};

namespace {

gs_status mlp_fail(gs_mlp* m, gs_status s, const std::string& msg) {
    if (m) m->err = msg;
    else global_fail(s, msg);
    return s;
}

gs_status mlp_cuda(gs_mlp* m, cudaError_t e, const char* what) {
    return mlp_fail(m, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
}

#define GS_MLPC(m, call)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return mlp_cuda((m), e_, #call); \
    } while (0)

gs_status ensure_partial(gs_mlp* m, int blocks) {
    if (blocks <= m->cap_blocks) return GS_OK;
    if (m->partial) {
        cudaStreamSynchronize(m->stream);
        cudaFree(m->partial);
        m->partial = nullptr;
        m->cap_blocks = 0;
    }
    GS_MLPC(m, gs_malloc(&m->partial, (size_t)blocks * PSTRIDE * sizeof(float)));
    m->cap_blocks = blocks;
    return GS_OK;
}

void fill_fwd(gs_mlp* m, const float* X, const float* y, long long row0, long long n, long long N, bool count,
              FwdBwdArgs* a) {
    a->params = m->params;
    a->mean = m->norm;
    a->inv_std = m->norm + NI;
    a->X = X;
    a->y = y;
    a->row0 = row0;
    a->n_rows = n;
    a->scale = 2.0f / (float)N;
    a->partial = m->partial;
    a->step = count ? m->step : nullptr;
}

void fill_red(gs_mlp* m, int blocks, float lr, bool update, ReduceAdamArgs* r) {
    r->partial = m->partial;
    r->n_blocks = blocks;
    r->grad = m->grad;
    r->loss = m->loss;
    r->params = m->params;
    r->m = m->m;
    r->v = m->v;
    r->step = m->step;
    r->lr = lr;
    r->update = update ? 1 : 0;
}

cudaError_t launch_pair(gs_mlp* m, const FwdBwdArgs& f, const ReduceAdamArgs& r, int blocks) {
    cudaError_t e = cudaFuncSetAttribute((const void*)mlp_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdBwdSmem);
    if (e != cudaSuccess) return e;
    mlp_fwd_bwd_kernel<<<blocks, ROWS, kFwdBwdSmem, m->stream>>>(f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp_reduce_adam_kernel<<<(NP + 1 + 255) / 256, 256, 0, m->stream>>>(r);
    return cudaGetLastError();
}

bool dev_ptr_ok(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

}  // namespace

extern "C" {

gs_status gs_mlp_create(gs_mlp** out, uint64_t seed, void* stream) {
    if (!out) return global_fail(GS_ERR_INVALID_ARG, "gs_mlp_create: out is NULL");
    *out = nullptr;
    gs_mlp* m = new (std::nothrow) gs_mlp();
    if (!m) return global_fail(GS_ERR_OOM, "gs_mlp_create: host allocation failed");
    cudaError_t e = cudaSuccess;
    if (stream) {
        m->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        m->own_stream = (e == cudaSuccess);
    }
    if (e == cudaSuccess) e = gs_malloc(&m->params, NP * sizeof(float));
    if (e == cudaSuccess) e = gs_malloc(&m->m, NP * sizeof(float));
    if (e == cudaSuccess) e = gs_malloc(&m->v, NP * sizeof(float));
    if (e == cudaSuccess) e = gs_malloc(&m->grad, NP * sizeof(float));
    if (e == cudaSuccess) e = gs_malloc(&m->norm, 2 * NI * sizeof(float));
    if (e == cudaSuccess) e = gs_malloc(&m->loss, sizeof(float));
    if (e == cudaSuccess) e = gs_malloc(&m->step, sizeof(long long));
    if (e == cudaSuccess) e = gs_malloc(&m->amin_idx, sizeof(long long));
    if (e == cudaSuccess) e = gs_malloc(&m->amin_val, sizeof(float));
    if (e != cudaSuccess) {
        gs_status st = mlp_cuda(nullptr, e, "gs_mlp_create");
        gs_mlp_destroy(m);
        return st;
    }
    // Glorot-uniform weights from splitmix64, zero biases, identity scaling.
    std::vector<float> p(NP, 0.f);
    uint64_t s = seed;
    auto fill = [&](int off, int fan_out, int fan_in) {
        const double lim = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) {
            const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            p[off + i] = (float)((2.0 * u - 1.0) * lim);
        }
    };
    fill(OW1, NH, NI);
    fill(OW2, NH, NH);
    fill(OW3, 1, NH);
    std::vector<float> norm(2 * NI);
    for (int k = 0; k < NI; ++k) {
        norm[k] = 0.f;
        norm[NI + k] = 1.f;
    }
    gs_status st = gs_mlp_set_params(m, p.data(), NP);
    if (st == GS_OK) {
        e = cudaMemcpyAsync(m->norm, norm.data(), norm.size() * sizeof(float), cudaMemcpyHostToDevice, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = mlp_cuda(nullptr, e, "gs_mlp_create");
    }
    if (st != GS_OK) {
        gs_mlp_destroy(m);
        return st;
    }
    *out = m;
    return GS_OK;
}

gs_status gs_mlp_destroy(gs_mlp* m) {
    if (!m) return GS_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void* p : {(void*)m->params, (void*)m->m, (void*)m->v, (void*)m->grad, (void*)m->norm, (void*)m->loss,
                    (void*)m->step, (void*)m->partial, (void*)m->pred, (void*)m->amin_idx, (void*)m->amin_val})
        if (p) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return GS_OK;
}

const char* gs_mlp_last_error(const gs_mlp* m) { return m ? m->err.c_str() : ""; }

gs_status gs_mlp_set_params(gs_mlp* m, const float* host, int64_t n) {
    if (!m || !host || n != NP) return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_set_params: need GS_MLP_PARAMS (1697) floats");
    GS_MLPC(m, cudaMemcpyAsync(m->params, host, NP * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    GS_MLPC(m, cudaMemsetAsync(m->m, 0, NP * sizeof(float), m->stream));
    GS_MLPC(m, cudaMemsetAsync(m->v, 0, NP * sizeof(float), m->stream));
    GS_MLPC(m, cudaMemsetAsync(m->step, 0, sizeof(long long), m->stream));
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    return GS_OK;
}

gs_status gs_mlp_get_params(gs_mlp* m, float* host, int64_t n) {
    if (!m || !host || n != NP) return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_get_params: need GS_MLP_PARAMS (1697) floats");
    GS_MLPC(m, cudaMemcpyAsync(host, m->params, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    return GS_OK;
}

gs_status gs_mlp_set_normalization(gs_mlp* m, const float* mean, const float* inv_std) {
    if (!m || !mean || !inv_std) return mlp_fail(m, GS_ERR_INVALID_ARG, "NULL argument");
    GS_MLPC(m, cudaMemcpyAsync(m->norm, mean, NI * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    GS_MLPC(m, cudaMemcpyAsync(m->norm + NI, inv_std, NI * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    return GS_OK;
}

gs_status gs_mlp_get_normalization(gs_mlp* m, float* mean, float* inv_std) {
    if (!m || !mean || !inv_std) return mlp_fail(m, GS_ERR_INVALID_ARG, "NULL argument");
    GS_MLPC(m, cudaMemcpyAsync(mean, m->norm, NI * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    GS_MLPC(m, cudaMemcpyAsync(inv_std, m->norm + NI, NI * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    return GS_OK;
}

gs_status gs_mlp_fit_normalization(gs_mlp* m, const float* X, int64_t n_rows) {
    if (!m || !dev_ptr_ok(X) || n_rows < 1) return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_fit_normalization: bad args");
    norm_kernel<<<NI, 256, 0, m->stream>>>(X, n_rows, m->norm, m->norm + NI);
    GS_MLPC(m, cudaGetLastError());
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    return GS_OK;
}

gs_status gs_mlp_loss_grad(gs_mlp* m, const float* X, const float* y, int64_t n_rows, float* loss_out,
                           float* grad_host) {
    if (!m || !dev_ptr_ok(X) || !dev_ptr_ok(y) || n_rows < 1)
        return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_loss_grad: bad args");
    const int blocks = (int)((n_rows + ROWS - 1) / ROWS);
    gs_status st = ensure_partial(m, blocks);
    if (st != GS_OK) return st;
    FwdBwdArgs f;
    ReduceAdamArgs r;
    fill_fwd(m, X, y, 0, n_rows, n_rows, false, &f);
    fill_red(m, blocks, 0.f, false, &r);
    GS_MLPC(m, launch_pair(m, f, r, blocks));
    float loss = 0.f;
    GS_MLPC(m, cudaMemcpyAsync(&loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (grad_host) GS_MLPC(m, cudaMemcpyAsync(grad_host, m->grad, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    if (loss_out) *loss_out = loss / (float)n_rows;
    return GS_OK;
}

gs_status gs_mlp_train(gs_mlp* m, const float* X, const float* y, int64_t n_rows, int32_t epochs,
                       int32_t batch_rows, float lr, float* final_loss) {
    if (!m || !dev_ptr_ok(X) || !dev_ptr_ok(y) || n_rows < 1 || epochs < 0 || batch_rows < 1 || !(lr > 0))
        return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_train: bad args");
    const int64_t nb = (n_rows + batch_rows - 1) / batch_rows;
    const int blocks = (int)((std::min<int64_t>(batch_rows, n_rows) + ROWS - 1) / ROWS);
    gs_status st = ensure_partial(m, blocks);
    if (st != GS_OK) return st;
    GS_MLPC(m, cudaFuncSetAttribute((const void*)mlp_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kFwdBwdSmem));
    // One epoch = nb minibatches in order, 2 kernel nodes each, built as a
    // linear graph and replayed once per epoch.
    cudaGraph_t g = nullptr;
    GS_MLPC(m, cudaGraphCreate(&g, 0));
    cudaGraphNode_t prev = nullptr;
    cudaError_t e = cudaSuccess;
    std::vector<FwdBwdArgs> fa(nb);
    std::vector<ReduceAdamArgs> ra(nb);
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
        const int64_t r0 = b * batch_rows;
        const int64_t n = std::min<int64_t>(batch_rows, n_rows - r0);
        const int bl = (int)((n + ROWS - 1) / ROWS);
        fill_fwd(m, X, y, r0, n, n, true, &fa[b]);
        fill_red(m, bl, lr, true, &ra[b]);
        void* a1[1] = {&fa[b]};
        void* a2[1] = {&ra[b]};
        cudaKernelNodeParams p1{};
        p1.func = (void*)mlp_fwd_bwd_kernel;
        p1.gridDim = dim3(bl);
        p1.blockDim = dim3(ROWS);
        p1.sharedMemBytes = (unsigned)kFwdBwdSmem;
        p1.kernelParams = a1;
        cudaKernelNodeParams p2{};
        p2.func = (void*)mlp_reduce_adam_kernel;
        p2.gridDim = dim3((NP + 1 + 255) / 256);
        p2.blockDim = dim3(256);
        p2.kernelParams = a2;
        cudaGraphNode_t n1, n2;
        e = gs_graph_add_kernel_node(&n1, g, prev ? &prev : nullptr, prev ? 1 : 0, &p1);
        if (e == cudaSuccess) e = gs_graph_add_kernel_node(&n2, g, &n1, 1, &p2);
        prev = n2;
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiateWithFlags(&ex, g, 0);
    if (e == cudaSuccess) e = cudaGraphUpload(ex, m->stream);
    for (int32_t ep = 0; ep < epochs && e == cudaSuccess; ++ep) e = cudaGraphLaunch(ex, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (ex) cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return mlp_cuda(m, e, "gs_mlp_train");
    if (final_loss) return gs_mlp_loss_grad(m, X, y, n_rows, final_loss, nullptr);
    return GS_OK;
}

gs_status gs_mlp_predict(gs_mlp* m, const float* X, int64_t n_rows, float* pred) {
    if (!m || !dev_ptr_ok(X) || !dev_ptr_ok(pred) || n_rows < 1)
        return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_predict: bad args");
    mlp_predict_kernel<false><<<(unsigned)((n_rows + 255) / 256), 256, 0, m->stream>>>(m->params, m->norm,
                                                                                     m->norm + NI, X, n_rows, pred);
    GS_MLPC(m, cudaGetLastError());
    return GS_OK;
}

namespace {

gs_status ensure_pred(gs_mlp* m, int64_t n_rows) {
    if (n_rows <= m->pred_cap) return GS_OK;
    if (m->pred) {
        cudaStreamSynchronize(m->stream);
        cudaFree(m->pred);
        m->pred = nullptr;
        m->pred_cap = 0;
    }
    GS_MLPC(m, gs_malloc(&m->pred, (size_t)n_rows * sizeof(float)));
    m->pred_cap = n_rows;
    return GS_OK;
}

gs_status finish_argmin(gs_mlp* m, int64_t n_rows, float scale, int64_t* best_row, float* best_pred) {
    argmin_kernel<<<1, 1024, 0, m->stream>>>(m->pred, n_rows, m->amin_idx, m->amin_val);
    GS_MLPC(m, cudaGetLastError());
    long long idx = -1;
    float val = 0.f;
    GS_MLPC(m, cudaMemcpyAsync(&idx, m->amin_idx, sizeof(idx), cudaMemcpyDeviceToHost, m->stream));
    GS_MLPC(m, cudaMemcpyAsync(&val, m->amin_val, sizeof(val), cudaMemcpyDeviceToHost, m->stream));
    GS_MLPC(m, cudaStreamSynchronize(m->stream));
    *best_row = idx;
    if (best_pred) *best_pred = val * scale;
    return GS_OK;
}

}  // namespace

gs_status gs_mlp_argmin(gs_mlp* m, const float* X, int64_t n_rows, int64_t* best_row, float* best_pred) {
    if (!m || !dev_ptr_ok(X) || n_rows < 1 || !best_row)
        return mlp_fail(m, GS_ERR_INVALID_ARG, "gs_mlp_argmin: bad args");
    gs_status st = ensure_pred(m, n_rows);
    if (st == GS_OK) st = gs_mlp_predict(m, X, n_rows, m->pred);
    if (st != GS_OK) return st;
    return finish_argmin(m, n_rows, 1.0f, best_row, best_pred);
}

gs_status gs_mlp_argmin_ensemble(gs_mlp* const* models, int32_t k, const float* X, int64_t n_rows,
                                 int64_t* best_row, float* best_pred) {
    if (!models || k < 1 || !dev_ptr_ok(X) || n_rows < 1 || !best_row)
        return mlp_fail(nullptr, GS_ERR_INVALID_ARG, "gs_mlp_argmin_ensemble: bad args");
    for (int32_t i = 0; i < k; ++i)
        if (!models[i]) return mlp_fail(nullptr, GS_ERR_INVALID_ARG, "gs_mlp_argmin_ensemble: NULL model");
    gs_mlp* m0 = models[0];
    for (int32_t i = 1; i < k; ++i) GS_MLPC(m0, cudaStreamSynchronize(models[i]->stream));
    gs_status st = ensure_pred(m0, n_rows);
    if (st != GS_OK) return st;
    const unsigned grid = (unsigned)((n_rows + 255) / 256);
    // sum of the members' predictions in member order, on the first member's stream
    for (int32_t i = 0; i < k; ++i) {
        const gs_mlp* mi = models[i];
        if (i == 0)
            mlp_predict_kernel<false><<<grid, 256, 0, m0->stream>>>(mi->params, mi->norm, mi->norm + NI, X, n_rows,
                                                                    m0->pred);
        else
            mlp_predict_kernel<true><<<grid, 256, 0, m0->stream>>>(mi->params, mi->norm, mi->norm + NI, X, n_rows,
                                                                   m0->pred);
        GS_MLPC(m0, cudaGetLastError());
    }
    return finish_argmin(m0, n_rows, 1.0f / (float)k, best_row, best_pred);
}

gs_status gs_features(const gs_workload* w, const gs_tune_candidate* c, int32_t n, float* out) {
    if (!w || !c || !out || n < 1) return global_fail(GS_ERR_INVALID_ARG, "gs_features: bad arguments");
    if (w->kind < GS_HEAT2D || w->kind > GS_FDTD3D || w->dtype < GS_F32 || w->dtype > GS_F16 || w->nx < 1 ||
        w->ny < 1 || w->nz < 1 || w->n_iters < 1)
        return global_fail(GS_ERR_INVALID_ARG, "gs_features: bad workload");
    for (int32_t i = 0; i < n; ++i) {
        const gs_plan& p = c[i].plan;
        if (c[i].batch_size < 0 || p.block_x < 1 || p.rows < 1 || p.temporal_depth < 1)
            return global_fail(GS_ERR_INVALID_ARG,
                               "gs_features: candidate " + std::to_string(i) +
                                   " needs explicit block_x, rows, temporal_depth and batch_size >= 0");
        float* f = out + (size_t)i * NI;
        f[0] = (float)std::log2((double)w->nx);
        f[1] = (float)std::log2((double)w->ny);
        f[2] = (float)std::log2((double)w->nz);
        f[3] = w->kind == GS_HEAT2D;
        f[4] = w->kind == GS_HEAT3D;
        f[5] = w->kind == GS_FDTD3D;
        // kernels per iteration: FDTD runs H and E as two launches, or one
        // fused launch
        f[6] = (w->kind == GS_FDTD3D && p.kernel != GS_KERNEL_FUSED) ? 2.f : 1.f;
        f[7] = (float)std::log2((double)w->n_iters);
        f[8] = w->dtype == GS_F32;
        f[9] = w->dtype == GS_BF16;
        f[10] = w->dtype == GS_F16;
        f[11] = c[i].batch_size > 0 ? (float)std::log2((double)c[i].batch_size) : 0.f;
        f[12] = c[i].batch_size == 0;
        f[13] = (float)std::log2((double)p.block_x);
        f[14] = (float)std::log2((double)p.rows);
        f[15] = (float)p.temporal_depth;
        // kernel variant, with AUTO resolved as the context resolves it
        int k = p.kernel;
        if (k == GS_KERNEL_AUTO) {
            k = (p.temporal_depth == 1 || w->kind == GS_HEAT2D)
                    ? GS_KERNEL_COLUMN
                    : (w->nz <= kWaveMaxNz ? GS_KERNEL_WAVE : GS_KERNEL_TILE);
        }
        f[16] = (k == GS_KERNEL_COLUMN || k == GS_KERNEL_COLUMN_SMEM);
        f[17] = (k == GS_KERNEL_COLUMN_SMEM);
    }
    return GS_OK;
}

// ------------------------------------------------ choosing a candidate --

}  // extern "C"

namespace {

// Batch sizes of the candidate set: per-step launch (0) and the graph batch
// sizes the paper sweeps (Sec. IV).
constexpr int64_t kPickBatchSizes[] = {0, 1, 10, 50, 100, 500, 1000};

gs_plan plan_of(int32_t block_x, int32_t rows, int32_t depth, int32_t kernel, int32_t tile_y = 0) {
    gs_plan p{};
    p.block_x = block_x;
    p.rows = rows;
    p.temporal_depth = depth;
    p.kernel = kernel;
    p.tile_y = tile_y;
    return p;
}

bool same_shape(const gs_plan& a, const gs_plan& b) {
    return a.block_x == b.block_x && a.rows == b.rows && a.temporal_depth == b.temporal_depth &&
           a.kernel == b.kernel && a.tile_y == b.tile_y;
}

// The launch plans the pickers (and the cost model's sweep) consider for a
// workload, in sweep order.  FDTD: COLUMN with 1, 2, 4, 8 rows, two
// k-march shapes and the fused step's k march (8 planes a block) with 4 and
// 8 rows.  Thermal: COLUMN with 2, 4, 8 rows; COLUMN_SMEM (2D and
// stacks of at most 8 planes); three MARCH shapes; WAVE at depth 2 and 4
// (2D and stacks of at most 16 planes); COLUMN at depth 2 and 4 (2D and
// stacks of at most 8 planes).  The library's default plan is included.
std::vector<gs_plan> candidate_plans(const gs_workload& w) {
    const int C = GS_KERNEL_COLUMN, CS = GS_KERNEL_COLUMN_SMEM, M = GS_KERNEL_MARCH, W = GS_KERNEL_WAVE;
    std::vector<gs_plan> v;
    gs_plan dflt;
    if (w.kind == GS_FDTD3D) {
        for (int32_t r : {1, 2, 4, 8}) v.push_back(plan_of(64, r, 1, C));
        v.push_back(plan_of(64, 4, 1, M));
        v.push_back(plan_of(32, 16, 1, M));
        for (int32_t r : {4, 8}) v.push_back(plan_of(64, r, 1, GS_KERNEL_FUSED, 8));
        dflt = plan_of(64, 4, 1, C);
    } else {
        const bool is2d = w.kind == GS_HEAT2D;
        for (int32_t r : {2, 4, 8}) v.push_back(plan_of(64, r, 1, C));
        if (is2d || w.nz <= 8)
            for (int32_t r : {4, 8}) v.push_back(plan_of(64, r, 1, CS));
        v.push_back(plan_of(32, 4, 1, M));
        v.push_back(plan_of(64, 8, 1, M));
        v.push_back(plan_of(32, 16, 1, M));
        if (is2d || w.nz <= 16) {
            for (int32_t t : {2, 4}) v.push_back(plan_of(64, 4, t, W));
            v.push_back(plan_of(64, 16, 4, W));
            for (int32_t t : {2, 4}) v.push_back(plan_of(128, 32, t, W));
        }
        if (is2d || w.nz <= 8)
            for (int32_t t : {2, 4}) v.push_back(plan_of(64, 4, t, C));
        const bool small = w.nx * w.ny * w.nz <= (int64_t(1) << 22);
        const bool deep = w.kind == GS_HEAT3D && w.nz > 8;
        dflt = plan_of(64, (small || deep) ? 4 : 8, 1, C);
    }
    bool have = false;
    for (const gs_plan& p : v) have = have || same_shape(p, dflt);
    if (!have) v.push_back(dflt);
    return v;
}

}  // namespace

extern "C" {

gs_status gs_candidates(const gs_workload* w, gs_tune_candidate* out, int32_t capacity, int32_t* n_out) {
    if (!w || !n_out || capacity < 0 || (capacity > 0 && !out))
        return global_fail(GS_ERR_INVALID_ARG, "gs_candidates: bad arguments");
    if (w->kind != GS_HEAT2D && w->kind != GS_HEAT3D && w->kind != GS_FDTD3D)
        return global_fail(GS_ERR_INVALID_ARG, "gs_candidates: kind must be GS_HEAT2D, GS_HEAT3D or GS_FDTD3D");
    const std::vector<gs_plan> plans = candidate_plans(*w);
    const int32_t nS = (int32_t)(sizeof(kPickBatchSizes) / sizeof(kPickBatchSizes[0]));
    const int32_t n = (int32_t)plans.size() * nS;
    *n_out = n;
    if (!out) return GS_OK;
    if (capacity < n) return global_fail(GS_ERR_INVALID_ARG, "gs_candidates: capacity below the candidate count");
    int32_t i = 0;
    for (const gs_plan& p : plans)
        for (int32_t k = 0; k < nS; ++k) {
            out[i].plan = p;
            out[i].batch_size = kPickBatchSizes[k];
            ++i;
        }
    return GS_OK;
}

}  // extern "C"

namespace {

// gs_pick over the candidates that `runnable` accepts (all when it is NULL).
gs_status pick_impl(gs_mlp* const* models, int32_t k, const gs_workload* w, bool (*runnable)(const gs_plan&),
                    gs_tune_candidate* best, float* pred_ms_per_iter) {
    if (!models || k < 1 || !w || !best) return global_fail(GS_ERR_INVALID_ARG, "gs_pick: bad arguments");
    for (int32_t i = 0; i < k; ++i)
        if (!models[i]) return global_fail(GS_ERR_INVALID_ARG, "gs_pick: NULL model");
    int32_t n = 0;
    gs_status st = gs_candidates(w, nullptr, 0, &n);
    if (st != GS_OK) return st;
    std::vector<gs_tune_candidate> all((size_t)n);
    st = gs_candidates(w, all.data(), n, &n);
    if (st != GS_OK) return st;
    // the candidates this grid can run (the checks gs_set_plan applies); the
    // refusals are expected, so the thread's last error message is kept
    const std::string saved = gs_last_error(nullptr);
    std::vector<gs_tune_candidate> ok;
    for (const gs_tune_candidate& c : all)
        if ((!runnable || runnable(c.plan)) && gs_plan_check(w, &c.plan, nullptr) == GS_OK) ok.push_back(c);
    global_fail(GS_OK, saved);
    if (ok.empty()) return global_fail(GS_ERR_UNSUPPORTED, "gs_pick: no candidate plan fits this grid");
    std::vector<float> X(ok.size() * (size_t)NI);
    st = gs_features(w, ok.data(), (int32_t)ok.size(), X.data());
    if (st != GS_OK) return st;
    gs_mlp* m0 = models[0];
    float* dX = nullptr;
    GS_MLPC(m0, gs_malloc(&dX, X.size() * sizeof(float)));
    // on the first model's stream, where the ensemble argmin runs
    cudaError_t e = cudaMemcpyAsync(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, m0->stream);
    int64_t row = -1;
    float pred = 0.f;
    if (e == cudaSuccess) st = gs_mlp_argmin_ensemble(models, k, dX, (int64_t)ok.size(), &row, &pred);
    const cudaError_t ef = cudaFree(dX);
    if (e != cudaSuccess) return mlp_cuda(m0, e, "gs_pick: feature upload");
    if (st != GS_OK) return st;
    if (ef != cudaSuccess) return mlp_cuda(m0, ef, "gs_pick: free");
    if (row < 0 || row >= (int64_t)ok.size()) return mlp_fail(m0, GS_ERR_NUMERIC, "gs_pick: no finite prediction");
    *best = ok[(size_t)row];
    if (pred_ms_per_iter) *pred_ms_per_iter = std::exp(pred);
    return GS_OK;
}

// FDTD in media runs on the COLUMN kernels and the fused march
bool media_runs(const gs_plan& p) {
    return p.kernel == GS_KERNEL_COLUMN || (p.kernel == GS_KERNEL_FUSED && p.tile_y >= 1);
}

}  // namespace

extern "C" {

gs_status gs_pick(gs_mlp* const* models, int32_t k, const gs_workload* w, gs_tune_candidate* best,
                  float* pred_ms_per_iter) {
    return pick_impl(models, k, w, nullptr, best, pred_ms_per_iter);
}

const char* gs_mlp_builtin_info(void) { return kBuiltinInfo; }

gs_status gs_mlp_create_builtin(gs_mlp** out, int32_t member, void* stream) {
    if (!out) return global_fail(GS_ERR_INVALID_ARG, "gs_mlp_create_builtin: out is NULL");
    *out = nullptr;
    if (member < 0 || member >= kBuiltinMembers)
        return global_fail(GS_ERR_INVALID_ARG, "gs_mlp_create_builtin: member must be in [0, " +
                                                   std::to_string(kBuiltinMembers) + ")");
    if (!kBuiltinTrained) return global_fail(GS_ERR_UNSUPPORTED, "gs_mlp_create_builtin: " + std::string(kBuiltinInfo));
    gs_mlp* m = nullptr;
    gs_status st = gs_mlp_create(&m, 0, stream);
    if (st != GS_OK) return st;
    st = gs_mlp_set_params(m, kBuiltinParams[member], NP);
    if (st == GS_OK) st = gs_mlp_set_normalization(m, kBuiltinNorm[member], kBuiltinNorm[member] + NI);
    if (st != GS_OK) {
        global_fail(st, "gs_mlp_create_builtin: " + m->err);
        gs_mlp_destroy(m);
        return st;
    }
    *out = m;
    return GS_OK;
}

gs_status gs_pick_ctx(gs_ctx* ctx, int64_t n_iters, gs_plan* plan_out, int64_t* batch_out, float* pred_ms_per_iter) {
    if (!ctx) return global_fail(GS_ERR_INVALID_ARG, "gs_pick_ctx: NULL context");
    if (!batch_out || n_iters < 1)
        return ctx_fail(ctx, GS_ERR_INVALID_ARG, "gs_pick_ctx: need batch_out and n_iters >= 1");
    gs_workload w;
    ctx_workload(ctx, &w);
    w.n_iters = n_iters;
    if (w.kind != GS_HEAT2D && w.kind != GS_HEAT3D && w.kind != GS_FDTD3D)
        return ctx_fail(ctx, GS_ERR_UNSUPPORTED, "gs_pick_ctx: the learned pick covers thermal and FDTD contexts");
    gs_mlp* models[kBuiltinMembers] = {};
    gs_status st = GS_OK;
    for (int k = 0; k < kBuiltinMembers && st == GS_OK; ++k)
        st = gs_mlp_create_builtin(&models[k], k, ctx_stream(ctx));
    gs_tune_candidate best{};
    std::string why;
    if (st == GS_OK) {
        st = pick_impl(models, kBuiltinMembers, &w, ctx_has_media(ctx) ? media_runs : nullptr, &best,
                       pred_ms_per_iter);
        if (st != GS_OK) why = models[0]->err.empty() ? gs_last_error(nullptr) : models[0]->err;
    } else {
        why = gs_last_error(nullptr);
    }
    for (gs_mlp* m : models) gs_mlp_destroy(m);
    if (st != GS_OK) return ctx_fail(ctx, st, "gs_pick_ctx: " + why);
    st = gs_set_plan(ctx, &best.plan);
    if (st != GS_OK) return st;  // message already on ctx
    if (plan_out) gs_get_plan(ctx, plan_out);
    *batch_out = best.batch_size;
    return GS_OK;
}

}  // extern "C"
