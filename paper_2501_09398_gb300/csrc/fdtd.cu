// Yee FDTD kernels: the paper's Maxwell solver launches one H-field kernel
// and one E-field kernel per time step (Sec. III-C).  Normalised units
// (eps = mu = c = 1, dx = 1), courant number s = dt:
//   H -= s*curl(E)  forward differences,
//   E += s*curl(H)  backward differences on interior unknowns only (PEC:
//                   tangential E on the walls is never written),
//   Ez[src] += amp*exp(-((n - delay)/width)^2)  soft source after E at step n.
// Staggering Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) Hx(i,j+1/2,k+1/2)
// Hy(i+1/2,j,k+1/2) Hz(i+1/2,j+1/2,k); each component is an (N+1)^2 x
// (Nk+1) array (Nk = N for the cube; the sub-domains of a slab set have
// their own Nk), row pitch >= N+1, indexed [k][j][i]; the walls k = 0 and
// k = Nk are PEC like the others.
//
// Each thread owns one 16-byte vector along i at fixed j and marches a
// chunk of kc planes in k, carrying the plane it needs from the previous
// step of the march (E at k+1 becomes E at k in the H kernel; H at k
// becomes H at k-1 in the E kernel).  i-neighbours come from warp shuffles
// (lane 31 / lane 0 load one scalar); j-neighbours are re-read (L1/L2).
#include <algorithm>

#define GS_CHECK_THIS_UNIT  // checked builds bounds-check this unit's field accesses
#include "common.cuh"

namespace gs {

enum { EX = 0, EY = 1, EZ = 2, HX = 3, HY = 4, HZ = 5 };

// Cells along i per thread of the column kernels, in every storage type.
constexpr int kFdtdColumnCells = 4;

// f -/+ s*((a - b) - (c - d)) with every rounding spelled out, so that both
// kernel variants produce the same bits.
__device__ __forceinline__ float curl_sub(float f, float s, float a, float b, float c, float d) {
    return __fmaf_rn(-s, __fsub_rn(__fsub_rn(a, b), __fsub_rn(c, d)), f);
}
__device__ __forceinline__ float curl_add(float f, float s, float a, float b, float c, float d) {
    return __fmaf_rn(s, __fsub_rn(__fsub_rn(a, b), __fsub_rn(c, d)), f);
}
// Media forms: da*f - db*curl and ca*f + cb*curl.  With a vacuum row
// (da = ca = 1, db = cb = s) they round exactly like curl_sub / curl_add.
__device__ __forceinline__ float curl_sub_m(float f, float2 m, float a, float b, float c, float d) {
    return __fmaf_rn(-m.y, __fsub_rn(__fsub_rn(a, b), __fsub_rn(c, d)), __fmul_rn(m.x, f));
}
__device__ __forceinline__ float curl_add_m(float f, float2 m, float a, float b, float c, float d) {
    return __fmaf_rn(m.y, __fsub_rn(__fsub_rn(a, b), __fsub_rn(c, d)), __fmul_rn(m.x, f));
}

// curl_sub / curl_add of two adjacent cells in Blackwell's packed FP32 pair
// operations (sub/fma .rn.f32x2), each half rounded as the scalar form
// rounds it, in the same order: ((a - b) - (c - d)), then the fused
// multiply-add.  An operand pair is two adjacent cells of a register array;
// a difference whose operands are shifted by one cell (an i-neighbour) is
// formed by scalar subtractions and passed in as a pair.
namespace {
__device__ __forceinline__ unsigned long long p2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void p2_out(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long p2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long p2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// sc * (t1 - t2) + f for a cell pair (sc = -s: curl_sub; s: curl_add)
__device__ __forceinline__ void curl2(const float* f, float sc, unsigned long long t1, unsigned long long t2, float* out) {
    p2_out(p2_fma(p2(sc, sc), p2_sub(t1, t2), p2(f[0], f[1])), out[0], out[1]);
}
// a - b for a cell pair of register arrays
__device__ __forceinline__ unsigned long long d2(const float* a, const float* b) {
    return p2_sub(p2(a[0], a[1]), p2(b[0], b[1]));
}
}  // namespace

template <typename ST>
__global__ void __launch_bounds__(256) fdtd_h_kernel(const FdtdArgs a) {
    constexpr int V = Vec<ST>::N;
    pdl_wait_then_trigger();
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const int lane = threadIdx.x & 31;
    const uint3 blk = block_index(a.rev);
    const int i0 = (blk.x * blockDim.x + threadIdx.x) * V;
    const int j = blk.y * blockDim.y + threadIdx.y;
    const int k0 = blk.z * a.kc;
    const int k1 = min(k0 + a.kc, Mk);
    const bool act = (i0 < M) && (j < M);
    const int nv = M - i0;  // valid elements in this vector (if act)
    const ST* Ex = static_cast<const ST*>(a.f[EX]);
    const ST* Ey = static_cast<const ST*>(a.f[EY]);
    const ST* Ez = static_cast<const ST*>(a.f[EZ]);
    ST* Hx = static_cast<ST*>(a.f[HX]);
    ST* Hy = static_cast<ST*>(a.f[HY]);
    ST* Hz = static_cast<ST*>(a.f[HZ]);
    const float s = a.s;
    const long long rowj = (long long)j * a.pitch + i0;

    float exk[V], eyk[V];
#pragma unroll
    for (int e = 0; e < V; ++e) { exk[e] = 0.f; eyk[e] = 0.f; }
    if (act) {
        load_vec(Ex + (long long)k0 * a.plane + rowj, exk);
        load_vec(Ey + (long long)k0 * a.plane + rowj, eyk);
    }
    for (int k = k0; k < k1; ++k) {
        const long long o = (long long)k * a.plane + rowj;
        float exk1[V], eyk1[V], ez[V], ezj1[V], exj1[V], hx[V], hy[V], hz[V];
#pragma unroll
        for (int e = 0; e < V; ++e) { exk1[e] = 0.f; eyk1[e] = 0.f; ez[e] = 0.f; ezj1[e] = 0.f; exj1[e] = 0.f; }
        float ez_r = 0.f, ey_r = 0.f;
        if (act) {
            if (k + 1 < Mk) {
                load_vec(Ex + o + a.plane, exk1);
                load_vec(Ey + o + a.plane, eyk1);
            }
            load_vec(Ez + o, ez);
            if (j + 1 < M) {
                load_vec(Ez + o + a.pitch, ezj1);
                load_vec(Ex + o + a.pitch, exj1);
            }
            load_vec_rw(Hx + o, hx);
            load_vec_rw(Hy + o, hy);
            load_vec_rw(Hz + o, hz);
            if (lane == 31 && i0 + V < M) {
                ez_r = load_scalar(Ez + o + V);
                ey_r = load_scalar(Ey + o + V);
            }
        }
        // i+1 neighbours of the last element come from the next lane.
        const float ez_n = __shfl_down_sync(0xffffffffu, ez[0], 1);
        const float ey_n = __shfl_down_sync(0xffffffffu, eyk[0], 1);
        if (act) {
            const float ez_last = (lane == 31) ? ez_r : ez_n;
            const float ey_last = (lane == 31) ? ey_r : ey_n;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int i = i0 + e;
                const float ez_ip = (e + 1 < V) ? ez[e + 1] : ez_last;
                const float ey_ip = (e + 1 < V) ? eyk[e + 1] : ey_last;
                if (j < N && k < Nk) hx[e] = curl_sub(hx[e], s, ezj1[e], ez[e], eyk1[e], eyk[e]);
                if (i < N && k < Nk) hy[e] = curl_sub(hy[e], s, exk1[e], exk[e], ez_ip, ez[e]);
                if (i < N && j < N) hz[e] = curl_sub(hz[e], s, ey_ip, eyk[e], exj1[e], exk[e]);
            }
            store_vec(Hx + o, hx, nv);
            store_vec(Hy + o, hy, nv);
            store_vec(Hz + o, hz, nv);
        }
#pragma unroll
        for (int e = 0; e < V; ++e) { exk[e] = exk1[e]; eyk[e] = eyk1[e]; }
    }
}

template <typename ST>
__global__ void __launch_bounds__(256) fdtd_e_kernel(const FdtdArgs a) {
    constexpr int V = Vec<ST>::N;
    pdl_wait_then_trigger();
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const int lane = threadIdx.x & 31;
    const uint3 blk = block_index(a.rev);
    const int i0 = (blk.x * blockDim.x + threadIdx.x) * V;
    const int j = blk.y * blockDim.y + threadIdx.y;
    const int k0 = blk.z * a.kc;
    const int k1 = min(k0 + a.kc, Mk);
    const bool act = (i0 < M) && (j < M);
    const int nv = M - i0;
    ST* Ex = static_cast<ST*>(a.f[EX]);
    ST* Ey = static_cast<ST*>(a.f[EY]);
    ST* Ez = static_cast<ST*>(a.f[EZ]);
    const ST* Hx = static_cast<const ST*>(a.f[HX]);
    const ST* Hy = static_cast<const ST*>(a.f[HY]);
    const ST* Hz = static_cast<const ST*>(a.f[HZ]);
    const float s = a.s;
    const long long rowj = (long long)j * a.pitch + i0;
    const bool j_int = (j >= 1 && j <= N - 1);

    float hxk_1[V], hyk_1[V];  // H at plane k-1
#pragma unroll
    for (int e = 0; e < V; ++e) { hxk_1[e] = 0.f; hyk_1[e] = 0.f; }
    if (act && k0 > 0) {
        load_vec(Hx + (long long)(k0 - 1) * a.plane + rowj, hxk_1);
        load_vec(Hy + (long long)(k0 - 1) * a.plane + rowj, hyk_1);
    }
    for (int k = k0; k < k1; ++k) {
        const long long o = (long long)k * a.plane + rowj;
        const bool k_int = (k >= 1 && k <= Nk - 1);
        float hx[V], hy[V], hz[V], hzj_1[V], hxj_1[V], ex[V], ey[V], ez[V];
#pragma unroll
        for (int e = 0; e < V; ++e) { hx[e] = 0.f; hy[e] = 0.f; hz[e] = 0.f; hzj_1[e] = 0.f; hxj_1[e] = 0.f; }
        float hz_l = 0.f, hy_l = 0.f;
        if (act) {
            load_vec(Hx + o, hx);
            load_vec(Hy + o, hy);
            load_vec(Hz + o, hz);
            if (j >= 1) {
                load_vec(Hz + o - a.pitch, hzj_1);
                load_vec(Hx + o - a.pitch, hxj_1);
            }
            load_vec_rw(Ex + o, ex);
            load_vec_rw(Ey + o, ey);
            load_vec_rw(Ez + o, ez);
            if (lane == 0 && i0 >= 1) {
                hz_l = load_scalar(Hz + o - 1);
                hy_l = load_scalar(Hy + o - 1);
            }
        }
        // i-1 neighbours of the first element come from the previous lane.
        const float hz_p = __shfl_up_sync(0xffffffffu, hz[V - 1], 1);
        const float hy_p = __shfl_up_sync(0xffffffffu, hy[V - 1], 1);
        if (act) {
            const float hz_first = (lane == 0) ? hz_l : hz_p;
            const float hy_first = (lane == 0) ? hy_l : hy_p;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int i = i0 + e;
                const bool i_int = (i >= 1 && i <= N - 1);
                const float hz_im = (e > 0) ? hz[e - 1] : hz_first;
                const float hy_im = (e > 0) ? hy[e - 1] : hy_first;
                if (i < N && j_int && k_int) ex[e] = curl_add(ex[e], s, hz[e], hzj_1[e], hy[e], hyk_1[e]);
                if (j < N && i_int && k_int) ey[e] = curl_add(ey[e], s, hx[e], hxk_1[e], hz[e], hz_im);
                if (k < Nk && i_int && j_int) ez[e] = curl_add(ez[e], s, hy[e], hy_im, hx[e], hxj_1[e]);
            }
            // The one thread that owns cell (si, sj, sk) keeps the device
            // step counter n and, if the source is on, adds it to Ez there.
            if (j == a.sj && k == a.sk && a.si >= i0 && a.si < i0 + V) {
                const long long n = *a.counter;
                if (a.src_on) {
                    const float u = __fdiv_rn(__fsub_rn((float)n, a.delay), a.width);
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (i0 + e == a.si) ez[e] = __fadd_rn(ez[e], __fmul_rn(a.amp, expf(-u * u)));
                }
                *a.counter = n + 1;
            }
            store_vec(Ex + o, ex, nv);
            store_vec(Ey + o, ey, nv);
            store_vec(Ez + o, ez, nv);
        }
#pragma unroll
        for (int e = 0; e < V; ++e) { hxk_1[e] = hx[e]; hyk_1[e] = hy[e]; }
    }
}

// ------------------------------------------------------------- column ----
//
// No march: each thread owns four cells along i (a 16-byte f32 or an 8-byte
// bf16/f16 access, so that a warp spans 128 cells in every storage type and
// N = 128, 256 take the aligned layout below) at one (j, k) and
// issues all of its loads at once (own components, the k+1 / j+1 (H) or
// k-1 / j-1 (E) neighbour vectors, and the i-edge scalars of lanes 31 / 0).
// Block (32, by, bz); neighbour vectors are re-read through L1/L2.
// MAT: lossy media; the thread also loads its vector of material ids with
// the fields and takes each cell's coefficients from the block's copy of
// the 256-row table in shared memory (staged once per block: through L1 the
// streaming field loads evict it and every lookup would wait on L2).
//
// Two bodies.  FAST serves the warps whose vectors all lie in [0, N) and
// whose (j, k) has every neighbour the update reads (H: j < N, k < Nk; E:
// 1 <= j <= N-1, 1 <= k <= Nk-1): all loads unconditional, no zero-filled registers, no
// per-cell predicates (E only keeps the i = 0 wall cell of lane 0).  The
// general body serves the rest with per-cell predicates.  ALN grids (N a
// multiple of the 32 V cells of a warp) cover only i in [0, N): the i = N
// column, where only Hx has an update, is an extra scalar cell of the lane
// 31 whose vector ends at i = N, in the last block along i (without it every
// (j, k) would need a second, one-cell warp); the lanes 31 of the other
// blocks end where the next block's lane 0 begins and own no extra cell.

// Ez[si, sj, sk] += source(n) and the step counter: the one thread that owns
// the source cell (in ALN grids with si = N, the lane 31 that owns the extra
// cell i = N) does both.
template <typename ST, int V, bool ALN>
__device__ __forceinline__ void fdtd_source(const FdtdArgs& a, int lane, int i0, int j, int k, long long o,
                                            float (&ez)[V], bool* extra_src) {
    *extra_src = false;
    if (j != a.sj || k != a.sk) return;
    const bool in_vec = (a.si >= i0 && a.si < i0 + V);
    const bool in_extra = ALN && lane == 31 && i0 + V == a.N && a.si == a.N;
    if (!in_vec && !in_extra) return;
    const long long n = *a.counter;
    if (a.src_on) {
        const float u = __fdiv_rn(__fsub_rn((float)n, a.delay), a.width);
        const float g = __fmul_rn(a.amp, expf(-u * u));
        if (in_vec) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (i0 + e == a.si) ez[e] = __fadd_rn(ez[e], g);
        } else {
            ST* Ez = static_cast<ST*>(a.f[EZ]);
            store_scalar(Ez + o + V, __fadd_rn(load_scalar_rw(Ez + o + V), g));
            *extra_src = true;
        }
    }
    *a.counter = n + 1;
}

template <typename ST, bool MAT, bool FAST, bool EXTRA>
__device__ __forceinline__ void fdtd_h_column_body(const FdtdArgs& a, const float2* s_med, int lane, int i0, int j,
                                                   int k) {
    constexpr int V = kFdtdColumnCells;
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const bool act = FAST || ((i0 < M) && (j < M) && (k < Mk));
    const ST* Ex = static_cast<const ST*>(a.f[EX]);
    const ST* Ey = static_cast<const ST*>(a.f[EY]);
    const ST* Ez = static_cast<const ST*>(a.f[EZ]);
    ST* Hx = static_cast<ST*>(a.f[HX]);
    ST* Hy = static_cast<ST*>(a.f[HY]);
    ST* Hz = static_cast<ST*>(a.f[HZ]);
    const float s = a.s;
    const long long o = act ? (long long)k * a.plane + (long long)j * a.pitch + i0 : 0;
    float exk[V], eyk[V], ez[V], exk1[V], eyk1[V], ezj1[V], exj1[V], hx[V], hy[V], hz[V];
    unsigned id[V];  // material ids (MAT), loaded with the fields
    float ez_r = 0.f, ey_r = 0.f;
    // lane 31's extra cell i = N (Hx only): Ez at j+1, Ey at k+1, Hx, id
    float ezj1_x = 0.f, eyk1_x = 0.f, hx_x = 0.f;
    unsigned id_x = 0;
    if constexpr (FAST) {
        if constexpr (MAT) load_ids<V>(a.mat + o, id);
        load_vecw<ST, V>(Ex + o, exk);
        load_vecw<ST, V>(Ey + o, eyk);
        load_vecw<ST, V>(Ez + o, ez);
        load_vecw<ST, V>(Ex + o + a.plane, exk1);
        load_vecw<ST, V>(Ey + o + a.plane, eyk1);
        load_vecw<ST, V>(Ez + o + a.pitch, ezj1);
        load_vecw<ST, V>(Ex + o + a.pitch, exj1);
        load_vecw_rw<ST, V>(Hx + o, hx);
        load_vecw_rw<ST, V>(Hy + o, hy);
        load_vecw_rw<ST, V>(Hz + o, hz);
        if (lane == 31) {  // i0 + V <= N: in range
            ez_r = load_scalar(Ez + o + V);
            ey_r = load_scalar(Ey + o + V);
            if constexpr (EXTRA) {
                ezj1_x = load_scalar(Ez + o + a.pitch + V);
                eyk1_x = load_scalar(Ey + o + a.plane + V);
                hx_x = load_scalar_rw(Hx + o + V);
                if constexpr (MAT) id_x = load_id(a.mat + o + V);
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) {
            exk[e] = 0.f; eyk[e] = 0.f; ez[e] = 0.f; exk1[e] = 0.f; eyk1[e] = 0.f; ezj1[e] = 0.f; exj1[e] = 0.f;
            hx[e] = 0.f; hy[e] = 0.f; hz[e] = 0.f;
            id[e] = 0;
        }
        if (act) {
            if constexpr (MAT) load_ids<V>(a.mat + o, id);
            load_vecw<ST, V>(Ex + o, exk);
            load_vecw<ST, V>(Ey + o, eyk);
            load_vecw<ST, V>(Ez + o, ez);
            if (k + 1 < Mk) {
                load_vecw<ST, V>(Ex + o + a.plane, exk1);
                load_vecw<ST, V>(Ey + o + a.plane, eyk1);
            }
            if (j + 1 < M) {
                load_vecw<ST, V>(Ez + o + a.pitch, ezj1);
                load_vecw<ST, V>(Ex + o + a.pitch, exj1);
            }
            load_vecw_rw<ST, V>(Hx + o, hx);
            load_vecw_rw<ST, V>(Hy + o, hy);
            load_vecw_rw<ST, V>(Hz + o, hz);
            if (lane == 31 && i0 + V < M) {
                ez_r = load_scalar(Ez + o + V);
                ey_r = load_scalar(Ey + o + V);
            }
        }
    }
    const float ez_n = __shfl_down_sync(0xffffffffu, ez[0], 1);
    const float ey_n = __shfl_down_sync(0xffffffffu, eyk[0], 1);
    if (!act) return;
    const float ez_last = (lane == 31) ? ez_r : ez_n;
    const float ey_last = (lane == 31) ? ey_r : ey_n;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = i0 + e;
        const float ez_ip = (e + 1 < V) ? ez[e + 1] : ez_last;
        const float ey_ip = (e + 1 < V) ? eyk[e + 1] : ey_last;
        const bool ux = FAST || (j < N && k < Nk);
        const bool uy = FAST || (i < N && k < Nk);
        const bool uz = FAST || (i < N && j < N);
        if constexpr (MAT) {
            const float2 m = s_med[id[e]];
            if (ux) hx[e] = curl_sub_m(hx[e], m, ezj1[e], ez[e], eyk1[e], eyk[e]);
            if (uy) hy[e] = curl_sub_m(hy[e], m, exk1[e], exk[e], ez_ip, ez[e]);
            if (uz) hz[e] = curl_sub_m(hz[e], m, ey_ip, eyk[e], exj1[e], exk[e]);
        } else {
            if (ux) hx[e] = curl_sub(hx[e], s, ezj1[e], ez[e], eyk1[e], eyk[e]);
            if (uy) hy[e] = curl_sub(hy[e], s, exk1[e], exk[e], ez_ip, ez[e]);
            if (uz) hz[e] = curl_sub(hz[e], s, ey_ip, eyk[e], exj1[e], exk[e]);
        }
    }
    const int nv = FAST ? V : M - i0;
    store_vecw<ST, V>(Hx + o, hx, nv);
    store_vecw<ST, V>(Hy + o, hy, nv);
    store_vecw<ST, V>(Hz + o, hz, nv);
    if constexpr (EXTRA) {
        if (lane == 31) {
            if constexpr (MAT) hx_x = curl_sub_m(hx_x, s_med[id_x], ezj1_x, ez_r, eyk1_x, ey_r);
            else hx_x = curl_sub(hx_x, s, ezj1_x, ez_r, eyk1_x, ey_r);
            store_scalar(Hx + o + V, hx_x);
        }
    }
}

template <typename ST, bool MAT, bool FAST, bool ALN>
__device__ __forceinline__ void fdtd_e_column_body(const FdtdArgs& a, const float2* s_med, int lane, int i0, int j,
                                                   int k) {
    constexpr int V = kFdtdColumnCells;
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const bool act = FAST || ((i0 < M) && (j < M) && (k < Mk));
    ST* Ex = static_cast<ST*>(a.f[EX]);
    ST* Ey = static_cast<ST*>(a.f[EY]);
    ST* Ez = static_cast<ST*>(a.f[EZ]);
    const ST* Hx = static_cast<const ST*>(a.f[HX]);
    const ST* Hy = static_cast<const ST*>(a.f[HY]);
    const ST* Hz = static_cast<const ST*>(a.f[HZ]);
    const float s = a.s;
    const long long o = act ? (long long)k * a.plane + (long long)j * a.pitch + i0 : 0;
    float hx[V], hy[V], hz[V], hxk_1[V], hyk_1[V], hzj_1[V], hxj_1[V], ex[V], ey[V], ez[V];
    unsigned id[V];  // material ids (MAT), loaded with the fields
    float hz_l = 0.f, hy_l = 0.f;
    if constexpr (FAST) {
        if constexpr (MAT) load_ids<V>(a.mat + o, id);
        load_vecw<ST, V>(Hx + o, hx);
        load_vecw<ST, V>(Hy + o, hy);
        load_vecw<ST, V>(Hz + o, hz);
        load_vecw<ST, V>(Hx + o - a.plane, hxk_1);
        load_vecw<ST, V>(Hy + o - a.plane, hyk_1);
        load_vecw<ST, V>(Hz + o - a.pitch, hzj_1);
        load_vecw<ST, V>(Hx + o - a.pitch, hxj_1);
        load_vecw_rw<ST, V>(Ex + o, ex);
        load_vecw_rw<ST, V>(Ey + o, ey);
        load_vecw_rw<ST, V>(Ez + o, ez);
        if (lane == 0) {  // the i = 0 cell's west value is never used: clamp the address
            const int dw = (i0 > 0) ? -1 : 0;
            hz_l = load_scalar(Hz + o + dw);
            hy_l = load_scalar(Hy + o + dw);
        }
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) {
            hx[e] = 0.f; hy[e] = 0.f; hz[e] = 0.f; hxk_1[e] = 0.f; hyk_1[e] = 0.f; hzj_1[e] = 0.f; hxj_1[e] = 0.f;
            ex[e] = 0.f; ey[e] = 0.f; ez[e] = 0.f;
            id[e] = 0;
        }
        if (act) {
            if constexpr (MAT) load_ids<V>(a.mat + o, id);
            load_vecw<ST, V>(Hx + o, hx);
            load_vecw<ST, V>(Hy + o, hy);
            load_vecw<ST, V>(Hz + o, hz);
            if (k >= 1) {
                load_vecw<ST, V>(Hx + o - a.plane, hxk_1);
                load_vecw<ST, V>(Hy + o - a.plane, hyk_1);
            }
            if (j >= 1) {
                load_vecw<ST, V>(Hz + o - a.pitch, hzj_1);
                load_vecw<ST, V>(Hx + o - a.pitch, hxj_1);
            }
            load_vecw_rw<ST, V>(Ex + o, ex);
            load_vecw_rw<ST, V>(Ey + o, ey);
            load_vecw_rw<ST, V>(Ez + o, ez);
            if (lane == 0 && i0 >= 1) {
                hz_l = load_scalar(Hz + o - 1);
                hy_l = load_scalar(Hy + o - 1);
            }
        }
    }
    const float hz_p = __shfl_up_sync(0xffffffffu, hz[V - 1], 1);
    const float hy_p = __shfl_up_sync(0xffffffffu, hy[V - 1], 1);
    if (!act) return;
    const float hz_first = (lane == 0) ? hz_l : hz_p;
    const float hy_first = (lane == 0) ? hy_l : hy_p;
    const bool j_int = FAST || (j >= 1 && j <= N - 1);
    const bool k_int = FAST || (k >= 1 && k <= Nk - 1);
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = i0 + e;
        // FAST: every i < N; only the i = 0 wall cell (lane 0 of the first warp) is not interior
        const bool i_int = FAST ? (e > 0 || i0 > 0) : (i >= 1 && i <= N - 1);
        const bool ux = FAST || (i < N && j_int && k_int);
        const bool uy = i_int && (FAST || (j < N && k_int));
        const bool uz = i_int && (FAST || (k < Nk && j_int));
        const float hz_im = (e > 0) ? hz[e - 1] : hz_first;
        const float hy_im = (e > 0) ? hy[e - 1] : hy_first;
        if constexpr (MAT) {
            const float2 m = s_med[id[e]];
            if (ux) ex[e] = curl_add_m(ex[e], m, hz[e], hzj_1[e], hy[e], hyk_1[e]);
            if (uy) ey[e] = curl_add_m(ey[e], m, hx[e], hxk_1[e], hz[e], hz_im);
            if (uz) ez[e] = curl_add_m(ez[e], m, hy[e], hy_im, hx[e], hxj_1[e]);
        } else {
            if (ux) ex[e] = curl_add(ex[e], s, hz[e], hzj_1[e], hy[e], hyk_1[e]);
            if (uy) ey[e] = curl_add(ey[e], s, hx[e], hxk_1[e], hz[e], hz_im);
            if (uz) ez[e] = curl_add(ez[e], s, hy[e], hy_im, hx[e], hxj_1[e]);
        }
    }
    bool extra_src;
    fdtd_source<ST, V, ALN>(a, lane, i0, j, k, o, ez, &extra_src);
    const int nv = FAST ? V : M - i0;
    store_vecw<ST, V>(Ex + o, ex, nv);
    store_vecw<ST, V>(Ey + o, ey, nv);
    store_vecw<ST, V>(Ez + o, ez, nv);
}

// Stage the media table (rows `base` .. base+255) in shared memory.
template <bool MAT>
__device__ __forceinline__ void stage_media(const FdtdArgs& a, float2* s_med, int base) {
    if constexpr (MAT) {
        const int nt = 32 * blockDim.y * blockDim.z;
        for (int t = threadIdx.x + 32 * (threadIdx.y + blockDim.y * threadIdx.z); t < 256; t += nt)
            s_med[t] = __ldg(a.med + base + t);
        __syncthreads();
    }
}

template <typename ST, bool MAT, bool ALN>
__global__ void __launch_bounds__(256, (MAT && sizeof(ST) == 4) ? 4 : 1) fdtd_h_column_kernel(const FdtdArgs a) {
    constexpr int V = kFdtdColumnCells;
    pdl_wait_then_trigger();
    __shared__ float2 s_med[MAT ? 256 : 1];
    stage_media<MAT>(a, s_med, 0);
    const int N = a.N;
    const int lane = threadIdx.x;
    const uint3 blk = block_index(a.rev);
    const int i0 = (blk.x * 32 + lane) * V;
    const int j = blk.y * blockDim.y + threadIdx.y;
    const int k = blk.z * blockDim.z + threadIdx.z;
    const bool in_x = ALN || __all_sync(0xffffffffu, i0 + V <= N);
    // EXTRA: the last block along i of an ALN grid, whose lane 31 ends at i = N
    if (in_x && j < N && k < a.Nk) {
        if (ALN && blk.x == gridDim.x - 1) fdtd_h_column_body<ST, MAT, true, true>(a, s_med, lane, i0, j, k);
        else fdtd_h_column_body<ST, MAT, true, false>(a, s_med, lane, i0, j, k);
    } else {
        fdtd_h_column_body<ST, MAT, false, false>(a, s_med, lane, i0, j, k);
    }
}

template <typename ST, bool MAT, bool ALN>
__global__ void __launch_bounds__(256, (MAT && sizeof(ST) == 4) ? 4 : 1) fdtd_e_column_kernel(const FdtdArgs a) {
    constexpr int V = kFdtdColumnCells;
    pdl_wait_then_trigger();
    __shared__ float2 s_med[MAT ? 256 : 1];
    stage_media<MAT>(a, s_med, 256);
    const int N = a.N;
    const int lane = threadIdx.x;
    const uint3 blk = block_index(a.rev);
    const int i0 = (blk.x * 32 + lane) * V;
    const int j = blk.y * blockDim.y + threadIdx.y;
    const int k = blk.z * blockDim.z + threadIdx.z;
    const bool in_x = ALN || __all_sync(0xffffffffu, i0 + V <= N);
    if (in_x && j >= 1 && j <= N - 1 && k >= 1 && k <= a.Nk - 1)
        fdtd_e_column_body<ST, MAT, true, ALN>(a, s_med, lane, i0, j, k);
    else
        fdtd_e_column_body<ST, MAT, false, ALN>(a, s_med, lane, i0, j, k);
}

// ------------------------------------------------------------- fused ----
//
// One Yee step per launch: H and E of the same cells in one pass, out of
// place (the state set a.f is read, the other set a.g written), so that no
// block overwrites a value a neighbouring block still reads.  Each thread
// owns four cells along i at one (j, k), as the column kernels.  It updates H
// on its cells from E^n; the E update then needs H^{n+1/2} also at j-1 (Hz,
// Hx), k-1 (Hy, Hx) and i-1 (Hz, Hy): the i-1 values come from the
// neighbouring lane (lane 0 recomputes its one cell), the j-1 and k-1 values
// are recomputed from E^n and H^{n-1/2} by the same rounded operations, on
// the same operands, as their owners' updates, so the step equals the H
// launch then the E launch bit for bit.  All six components are written to
// a.g, updated or not (the walls' fixed values included); the soft source
// is added to a.g's Ez.  Bytes per cell-step: six components read and six
// written, against nine and nine for the two launches.  Neighbour values
// come from loads at clamped offsets where they fall outside the arrays;
// such values are never used (the update masks exclude them).
// A value as a store to the storage type and a load back give it.
template <typename ST>
__device__ __forceinline__ float stored(float v) {
    return to_f32(from_f32<ST>(v));
}

template <typename ST, bool FAST, bool ALN>
__device__ __forceinline__ void fdtd_fused_body(const FdtdArgs& a, int lane, int i0, int j, int k) {
    constexpr int V = kFdtdColumnCells;
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const bool act = FAST || ((i0 < M) && (j < M) && (k < Mk));
    const long long P = a.pitch, PL = a.plane;
    // a thread past the arrays (act false) loads at offset 0 only
    const long long dj1 = (FAST || (act && j + 1 < M)) ? P : 0;
    const long long dk1 = (FAST || (act && k + 1 < Mk)) ? PL : 0;
    const long long djm = (FAST || (act && j >= 1)) ? -P : 0;
    const long long dkm = (FAST || (act && k >= 1)) ? -PL : 0;
    const long long o = act ? (long long)k * PL + (long long)j * P + i0 : 0;
    const ST* Ex = static_cast<const ST*>(a.f[EX]);
    const ST* Ey = static_cast<const ST*>(a.f[EY]);
    const ST* Ez = static_cast<const ST*>(a.f[EZ]);
    const ST* Hx = static_cast<const ST*>(a.f[HX]);
    const ST* Hy = static_cast<const ST*>(a.f[HY]);
    const ST* Hz = static_cast<const ST*>(a.f[HZ]);
    const float s = a.s;
    // own cells, the H update's j+1 / k+1 neighbours, and the rows j-1 and
    // planes k-1 whose H the E update needs
    float ex[V], ey[V], ez[V], hx[V], hy[V], hz[V], exk1[V], eyk1[V], ezj1[V], exj1[V];
    float hzjm[V], hxjm[V], eyjm[V], exjm[V], ezjm[V], eyjmk1[V];
    float hykm[V], hxkm[V], exkm[V], ezkm[V], eykm[V], ezj1km[V];
    load_vecw<ST, V>(Ex + o, ex);
    load_vecw<ST, V>(Ey + o, ey);
    load_vecw<ST, V>(Ez + o, ez);
    load_vecw<ST, V>(Hx + o, hx);
    load_vecw<ST, V>(Hy + o, hy);
    load_vecw<ST, V>(Hz + o, hz);
    load_vecw<ST, V>(Ex + o + dk1, exk1);
    load_vecw<ST, V>(Ey + o + dk1, eyk1);
    load_vecw<ST, V>(Ez + o + dj1, ezj1);
    load_vecw<ST, V>(Ex + o + dj1, exj1);
    load_vecw<ST, V>(Hz + o + djm, hzjm);
    load_vecw<ST, V>(Hx + o + djm, hxjm);
    load_vecw<ST, V>(Ey + o + djm, eyjm);
    load_vecw<ST, V>(Ex + o + djm, exjm);
    load_vecw<ST, V>(Ez + o + djm, ezjm);
    load_vecw<ST, V>(Ey + o + djm + dk1, eyjmk1);
    load_vecw<ST, V>(Hy + o + dkm, hykm);
    load_vecw<ST, V>(Hx + o + dkm, hxkm);
    load_vecw<ST, V>(Ex + o + dkm, exkm);
    load_vecw<ST, V>(Ez + o + dkm, ezkm);
    load_vecw<ST, V>(Ey + o + dkm, eykm);
    load_vecw<ST, V>(Ez + o + dkm + dj1, ezj1km);
    // i+1 neighbours of lane 31's last cell (the next warp's first): Ez, Ey
    // at (j, k), Ey at j-1, Ez at k-1; and, in ALN grids, what the i = N
    // cell's Hx update reads
    const bool has_r = (lane == 31) && (FAST || (act && i0 + V < M));
    float ez_r = 0.f, ey_r = 0.f, eyjm_r = 0.f, ezkm_r = 0.f, ezj1_x = 0.f, eyk1_x = 0.f;
    if (has_r) {
        ez_r = load_scalar(Ez + o + V);
        ey_r = load_scalar(Ey + o + V);
        eyjm_r = load_scalar(Ey + o + djm + V);
        ezkm_r = load_scalar(Ez + o + dkm + V);
        if (ALN && i0 + V == N) {
            ezj1_x = load_scalar(Ez + o + dj1 + V);
            eyk1_x = load_scalar(Ey + o + dk1 + V);
        }
    }
    // lane 0's i-1 cell (the previous warp's last), for its H at i-1
    float hz_l = 0.f, hy_l = 0.f, ey_l = 0.f, ex_l = 0.f, ez_l = 0.f, exj1_l = 0.f, exk1_l = 0.f;
    if (lane == 0 && i0 >= 1 && act) {
        hz_l = load_scalar(Hz + o - 1);
        hy_l = load_scalar(Hy + o - 1);
        ey_l = load_scalar(Ey + o - 1);
        ex_l = load_scalar(Ex + o - 1);
        ez_l = load_scalar(Ez + o - 1);
        exj1_l = load_scalar(Ex + o + dj1 - 1);
        exk1_l = load_scalar(Ex + o + dk1 - 1);
    }
    const float ez_n = __shfl_down_sync(0xffffffffu, ez[0], 1);
    const float ey_n = __shfl_down_sync(0xffffffffu, ey[0], 1);
    const float eyjm_n = __shfl_down_sync(0xffffffffu, eyjm[0], 1);
    const float ezkm_n = __shfl_down_sync(0xffffffffu, ezkm[0], 1);
    const float ez_last = (lane == 31) ? ez_r : ez_n;
    const float ey_last = (lane == 31) ? ey_r : ey_n;
    const float eyjm_last = (lane == 31) ? eyjm_r : eyjm_n;
    const float ezkm_last = (lane == 31) ? ezkm_r : ezkm_n;

    // H^{n+1/2}: own cells, and the j-1 / k-1 values the E update reads
    float hxn[V], hyn[V], hzn[V], hzjmn[V], hxjmn[V], hykmn[V], hxkmn[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = i0 + e;
        const float ez_ip = (e + 1 < V) ? ez[e + 1] : ez_last;
        const float ey_ip = (e + 1 < V) ? ey[e + 1] : ey_last;
        const float eyjm_ip = (e + 1 < V) ? eyjm[e + 1] : eyjm_last;
        const float ezkm_ip = (e + 1 < V) ? ezkm[e + 1] : ezkm_last;
        const bool iN = FAST || i < N;
        hxn[e] = (FAST || (j < N && k < Nk)) ? curl_sub(hx[e], s, ezj1[e], ez[e], eyk1[e], ey[e]) : hx[e];
        hyn[e] = (FAST || (iN && k < Nk)) ? curl_sub(hy[e], s, exk1[e], ex[e], ez_ip, ez[e]) : hy[e];
        hzn[e] = (FAST || (iN && j < N)) ? curl_sub(hz[e], s, ey_ip, ey[e], exj1[e], ex[e]) : hz[e];
        // row j-1: its j+1 row is row j (own Ex, Ez); plane k-1: its k+1
        // plane is plane k (own Ex, Ey)
        hzjmn[e] = iN ? curl_sub(hzjm[e], s, eyjm_ip, eyjm[e], ex[e], exjm[e]) : hzjm[e];
        hxjmn[e] = (FAST || k < Nk) ? curl_sub(hxjm[e], s, ez[e], ezjm[e], eyjmk1[e], eyjm[e]) : hxjm[e];
        hykmn[e] = iN ? curl_sub(hykm[e], s, ex[e], exkm[e], ezkm_ip, ezkm[e]) : hykm[e];
        hxkmn[e] = (FAST || j < N) ? curl_sub(hxkm[e], s, ezj1km[e], ezkm[e], ey[e], eykm[e]) : hxkm[e];
        // the E launch of the two-launch step reads H as stored: round to
        // the storage type (identity for f32)
        hxn[e] = stored<ST>(hxn[e]);
        hyn[e] = stored<ST>(hyn[e]);
        hzn[e] = stored<ST>(hzn[e]);
        hzjmn[e] = stored<ST>(hzjmn[e]);
        hxjmn[e] = stored<ST>(hxjmn[e]);
        hykmn[e] = stored<ST>(hykmn[e]);
        hxkmn[e] = stored<ST>(hxkmn[e]);
    }
    // i-1: the previous lane's last cell; lane 0 recomputes its own
    float hz_first = __shfl_up_sync(0xffffffffu, hzn[V - 1], 1);
    float hy_first = __shfl_up_sync(0xffffffffu, hyn[V - 1], 1);
    if (lane == 0) {
        const int im = i0 - 1;  // < N whenever i0 <= N
        hz_first = stored<ST>((im >= 0 && (FAST || j < N)) ? curl_sub(hz_l, s, ey[0], ey_l, exj1_l, ex_l) : hz_l);
        hy_first = stored<ST>((im >= 0 && (FAST || k < Nk)) ? curl_sub(hy_l, s, exk1_l, ex_l, ez[0], ez_l) : hy_l);
    }
    if (!act) return;

    // E^{n+1}
    const bool j_int = FAST || (j >= 1 && j <= N - 1);
    const bool k_int = FAST || (k >= 1 && k <= Nk - 1);
    float exn[V], eyn[V], ezn[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = i0 + e;
        const bool i_int = FAST ? (e > 0 || i0 > 0) : (i >= 1 && i <= N - 1);
        const float hz_im = (e > 0) ? hzn[e - 1] : hz_first;
        const float hy_im = (e > 0) ? hyn[e - 1] : hy_first;
        exn[e] = ((FAST || i < N) && j_int && k_int) ? curl_add(ex[e], s, hzn[e], hzjmn[e], hyn[e], hykmn[e]) : ex[e];
        eyn[e] = ((FAST || j < N) && i_int && k_int) ? curl_add(ey[e], s, hxn[e], hxkmn[e], hzn[e], hz_im) : ey[e];
        ezn[e] = ((FAST || k < Nk) && i_int && j_int) ? curl_add(ez[e], s, hyn[e], hy_im, hxn[e], hxjmn[e]) : ez[e];
    }
    // lane 31's extra cell i = N (ALN): Hx is its one update; E, Hy, Hz copied
    float x_ex = 0.f, x_hx = 0.f, x_hy = 0.f, x_hz = 0.f, x_ez = ez_r;
    const bool xcell = ALN && lane == 31 && i0 + V == N;
    if (xcell) {
        x_ex = load_scalar(Ex + o + V);
        x_hx = load_scalar(Hx + o + V);
        x_hy = load_scalar(Hy + o + V);
        x_hz = load_scalar(Hz + o + V);
        if (FAST || (j < N && k < Nk)) x_hx = curl_sub(x_hx, s, ezj1_x, ez_r, eyk1_x, ey_r);
    }
    // the soft source on the new Ez, and the step counter
    if (j == a.sj && k == a.sk) {
        const bool in_vec = (a.si >= i0 && a.si < i0 + V);
        const bool in_extra = xcell && a.si == N;
        if (in_vec || in_extra) {
            const long long n = *a.counter;
            if (a.src_on) {
                const float u = __fdiv_rn(__fsub_rn((float)n, a.delay), a.width);
                const float gsrc = __fmul_rn(a.amp, expf(-u * u));
                if (in_vec) {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (i0 + e == a.si) ezn[e] = __fadd_rn(ezn[e], gsrc);
                } else {
                    x_ez = __fadd_rn(x_ez, gsrc);
                }
            }
            *a.counter = n + 1;
        }
    }
    const int nv = FAST ? V : M - i0;
    store_vecw<ST, V>(static_cast<ST*>(a.g[EX]) + o, exn, nv);
    store_vecw<ST, V>(static_cast<ST*>(a.g[EY]) + o, eyn, nv);
    store_vecw<ST, V>(static_cast<ST*>(a.g[EZ]) + o, ezn, nv);
    store_vecw<ST, V>(static_cast<ST*>(a.g[HX]) + o, hxn, nv);
    store_vecw<ST, V>(static_cast<ST*>(a.g[HY]) + o, hyn, nv);
    store_vecw<ST, V>(static_cast<ST*>(a.g[HZ]) + o, hzn, nv);
    if (xcell) {
        store_scalar(static_cast<ST*>(a.g[EX]) + o + V, x_ex);
        store_scalar(static_cast<ST*>(a.g[EY]) + o + V, ey_r);
        store_scalar(static_cast<ST*>(a.g[EZ]) + o + V, x_ez);
        store_scalar(static_cast<ST*>(a.g[HX]) + o + V, x_hx);
        store_scalar(static_cast<ST*>(a.g[HY]) + o + V, x_hy);
        store_scalar(static_cast<ST*>(a.g[HZ]) + o + V, x_hz);
    }
}

template <typename ST, bool ALN>
__global__ void __launch_bounds__(256, 2) fdtd_fused_kernel(const FdtdArgs a) {
    constexpr int V = kFdtdColumnCells;
    pdl_wait_then_trigger();
    const int N = a.N;
    const int lane = threadIdx.x;
    const uint3 blk = block_index(a.rev);
    const int i0 = (blk.x * 32 + lane) * V;
    const int j = blk.y * blockDim.y + threadIdx.y;
    const int k = blk.z * blockDim.z + threadIdx.z;
    const bool in_x = ALN || __all_sync(0xffffffffu, i0 + V <= N);
    if (in_x && j >= 1 && j <= N - 1 && k >= 1 && k <= a.Nk - 1)
        fdtd_fused_body<ST, true, ALN>(a, lane, i0, j, k);
    else
        fdtd_fused_body<ST, false, ALN>(a, lane, i0, j, k);
}

// The fused step marching in k.  A block of 32 x BY threads owns 128 cells
// along i (four a lane) x BY rows j x kmarch planes k and walks its planes
// upwards.  The E update of plane k reads H^{n+1/2} of plane k-1 (Hy, Hx),
// which the same thread computed on the plane before and keeps in registers
// (the column form recomputes it from six more loads); E^n of plane k+1,
// loaded for the H update, is E^n of plane k on the next plane, and Ey of
// row j-1 likewise.  The j-1 values of H^{n+1/2} (Hz, Hx) belong to another
// warp and are recomputed from loads, the i-1 values come from the
// neighbouring lane (lane 0 recomputes its one cell), as in the column form.
// Every value is formed by the same rounded operations on the same operands
// as in the two launches, so the result is the same bit for bit (interior
// warps in vacuum take the operations in packed pairs, each half rounded as
// the scalar form; in media each cell's coefficients come from the table
// rows the block holds in shared memory).  A block whose first plane k0 is
// above the wall recomputes H^{n+1/2} of plane k0-1 once before its march.
template <typename ST, bool FAST, bool ALN, bool MAT>
__device__ __forceinline__ void fdtd_march_plane(const FdtdArgs& a, const float2* s_mh, const float2* s_me, int lane,
                                                 int i0, bool act_i, int j, int k,
                                                 float (&ex)[kFdtdColumnCells], float (&ey)[kFdtdColumnCells],
                                                 float (&ez)[kFdtdColumnCells], float (&hykm)[kFdtdColumnCells],
                                                 float (&hxkm)[kFdtdColumnCells], float (&eyjm)[kFdtdColumnCells]) {
    constexpr int V = kFdtdColumnCells;
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const long long P = a.pitch, PL = a.plane;
    const long long dj1 = (FAST || j + 1 < M) ? P : 0;
    const long long dk1 = (FAST || k + 1 < Mk) ? PL : 0;
    const long long djm = (FAST || j >= 1) ? -P : 0;
    // lanes past the arrays (act_i false) load at the start of their row
    const long long o = (long long)k * PL + (long long)j * P + ((FAST || act_i) ? i0 : 0);
    const ST* Ex = static_cast<const ST*>(a.f[EX]);
    const ST* Ey = static_cast<const ST*>(a.f[EY]);
    const ST* Ez = static_cast<const ST*>(a.f[EZ]);
    const ST* Hx = static_cast<const ST*>(a.f[HX]);
    const ST* Hy = static_cast<const ST*>(a.f[HY]);
    const ST* Hz = static_cast<const ST*>(a.f[HZ]);
    const float s = a.s;
    float hx[V], hy[V], hz[V], ex1[V], ey1[V], ez1[V], ezj1[V], exj1[V];
    float hzjm[V], hxjm[V], exjm[V], ezjm[V], eyjm1[V];
    load_vecw<ST, V>(Hx + o, hx);
    load_vecw<ST, V>(Hy + o, hy);
    load_vecw<ST, V>(Hz + o, hz);
    load_vecw<ST, V>(Ex + o + dk1, ex1);
    load_vecw<ST, V>(Ey + o + dk1, ey1);
    load_vecw<ST, V>(Ez + o + dk1, ez1);
    load_vecw<ST, V>(Ez + o + dj1, ezj1);
    load_vecw<ST, V>(Ex + o + dj1, exj1);
    load_vecw<ST, V>(Hz + o + djm, hzjm);
    load_vecw<ST, V>(Hx + o + djm, hxjm);
    load_vecw<ST, V>(Ex + o + djm, exjm);
    load_vecw<ST, V>(Ez + o + djm, ezjm);
    load_vecw<ST, V>(Ey + o + djm + dk1, eyjm1);
    // media: the material ids of the own cells and of row j-1
    unsigned id[V], idjm[V];
    if constexpr (MAT) {
        load_ids<V>(a.mat + o, id);
        load_ids<V>(a.mat + o + djm, idjm);
    }
    // i+1 neighbours of lane 31's last cell; the aligned layout's i = N cell
    const bool has_r = (lane == 31) && (FAST || (act_i && i0 + V < M));
    float ez_r = 0.f, ey_r = 0.f, eyjm_r = 0.f, ezj1_x = 0.f, eyk1_x = 0.f;
    if (has_r) {
        ez_r = load_scalar(Ez + o + V);
        ey_r = load_scalar(Ey + o + V);
        eyjm_r = load_scalar(Ey + o + djm + V);
        if (ALN && i0 + V == N) {
            ezj1_x = load_scalar(Ez + o + dj1 + V);
            eyk1_x = load_scalar(Ey + o + dk1 + V);
        }
    }
    // lane 0's i-1 cell, for its H at i-1
    float hz_l = 0.f, hy_l = 0.f, ey_l = 0.f, ex_l = 0.f, ez_l = 0.f, exj1_l = 0.f, exk1_l = 0.f;
    unsigned id_l = 0;
    if (lane == 0 && i0 >= 1 && (FAST || act_i)) {
        if constexpr (MAT) id_l = load_id(a.mat + o - 1);
        hz_l = load_scalar(Hz + o - 1);
        hy_l = load_scalar(Hy + o - 1);
        ey_l = load_scalar(Ey + o - 1);
        ex_l = load_scalar(Ex + o - 1);
        ez_l = load_scalar(Ez + o - 1);
        exj1_l = load_scalar(Ex + o + dj1 - 1);
        exk1_l = load_scalar(Ex + o + dk1 - 1);
    }
    const float ez_n = __shfl_down_sync(0xffffffffu, ez[0], 1);
    const float ey_n = __shfl_down_sync(0xffffffffu, ey[0], 1);
    const float eyjm_n = __shfl_down_sync(0xffffffffu, eyjm[0], 1);
    const float ez_last = (lane == 31) ? ez_r : ez_n;
    const float ey_last = (lane == 31) ? ey_r : ey_n;
    const float eyjm_last = (lane == 31) ? eyjm_r : eyjm_n;

    // H^{n+1/2} of the own cells and of row j-1
    float hxn[V], hyn[V], hzn[V], hzjmn[V], hxjmn[V];
    if constexpr (FAST && !MAT) {
        // every cell updates: packed pairs; the i-shifted differences scalar
        float dz[V], dy[V], dyj[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            dz[e] = __fsub_rn((e + 1 < V) ? ez[e + 1] : ez_last, ez[e]);
            dy[e] = __fsub_rn((e + 1 < V) ? ey[e + 1] : ey_last, ey[e]);
            dyj[e] = __fsub_rn((e + 1 < V) ? eyjm[e + 1] : eyjm_last, eyjm[e]);
        }
#pragma unroll
        for (int e = 0; e < V; e += 2) {
            curl2(&hx[e], -s, d2(&ezj1[e], &ez[e]), d2(&ey1[e], &ey[e]), &hxn[e]);
            curl2(&hy[e], -s, d2(&ex1[e], &ex[e]), p2(dz[e], dz[e + 1]), &hyn[e]);
            curl2(&hz[e], -s, p2(dy[e], dy[e + 1]), d2(&exj1[e], &ex[e]), &hzn[e]);
            curl2(&hzjm[e], -s, p2(dyj[e], dyj[e + 1]), d2(&ex[e], &exjm[e]), &hzjmn[e]);
            curl2(&hxjm[e], -s, d2(&ez[e], &ezjm[e]), d2(&eyjm1[e], &eyjm[e]), &hxjmn[e]);
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
            hxn[e] = stored<ST>(hxn[e]);
            hyn[e] = stored<ST>(hyn[e]);
            hzn[e] = stored<ST>(hzn[e]);
            hzjmn[e] = stored<ST>(hzjmn[e]);
            hxjmn[e] = stored<ST>(hxjmn[e]);
        }
    } else
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = i0 + e;
        const float ez_ip = (e + 1 < V) ? ez[e + 1] : ez_last;
        const float ey_ip = (e + 1 < V) ? ey[e + 1] : ey_last;
        const float eyjm_ip = (e + 1 < V) ? eyjm[e + 1] : eyjm_last;
        const bool iN = FAST || i < N;
        if constexpr (MAT) {
            const float2 m = s_mh[id[e]], mj = s_mh[idjm[e]];
            hxn[e] = stored<ST>((FAST || (j < N && k < Nk)) ? curl_sub_m(hx[e], m, ezj1[e], ez[e], ey1[e], ey[e]) : hx[e]);
            hyn[e] = stored<ST>((FAST || (iN && k < Nk)) ? curl_sub_m(hy[e], m, ex1[e], ex[e], ez_ip, ez[e]) : hy[e]);
            hzn[e] = stored<ST>((FAST || (iN && j < N)) ? curl_sub_m(hz[e], m, ey_ip, ey[e], exj1[e], ex[e]) : hz[e]);
            hzjmn[e] = stored<ST>(iN ? curl_sub_m(hzjm[e], mj, eyjm_ip, eyjm[e], ex[e], exjm[e]) : hzjm[e]);
            hxjmn[e] = stored<ST>((FAST || k < Nk) ? curl_sub_m(hxjm[e], mj, ez[e], ezjm[e], eyjm1[e], eyjm[e]) : hxjm[e]);
        } else {
            hxn[e] = stored<ST>((FAST || (j < N && k < Nk)) ? curl_sub(hx[e], s, ezj1[e], ez[e], ey1[e], ey[e]) : hx[e]);
            hyn[e] = stored<ST>((FAST || (iN && k < Nk)) ? curl_sub(hy[e], s, ex1[e], ex[e], ez_ip, ez[e]) : hy[e]);
            hzn[e] = stored<ST>((FAST || (iN && j < N)) ? curl_sub(hz[e], s, ey_ip, ey[e], exj1[e], ex[e]) : hz[e]);
            hzjmn[e] = stored<ST>(iN ? curl_sub(hzjm[e], s, eyjm_ip, eyjm[e], ex[e], exjm[e]) : hzjm[e]);
            hxjmn[e] = stored<ST>((FAST || k < Nk) ? curl_sub(hxjm[e], s, ez[e], ezjm[e], eyjm1[e], eyjm[e]) : hxjm[e]);
        }
    }
    float hz_first = __shfl_up_sync(0xffffffffu, hzn[V - 1], 1);
    float hy_first = __shfl_up_sync(0xffffffffu, hyn[V - 1], 1);
    if (lane == 0) {
        const int im = i0 - 1;
        if constexpr (MAT) {
            const float2 m = s_mh[id_l];
            hz_first = stored<ST>((im >= 0 && (FAST || j < N)) ? curl_sub_m(hz_l, m, ey[0], ey_l, exj1_l, ex_l) : hz_l);
            hy_first = stored<ST>((im >= 0 && (FAST || k < Nk)) ? curl_sub_m(hy_l, m, exk1_l, ex_l, ez[0], ez_l) : hy_l);
        } else {
            hz_first = stored<ST>((im >= 0 && (FAST || j < N)) ? curl_sub(hz_l, s, ey[0], ey_l, exj1_l, ex_l) : hz_l);
            hy_first = stored<ST>((im >= 0 && (FAST || k < Nk)) ? curl_sub(hy_l, s, exk1_l, ex_l, ez[0], ez_l) : hy_l);
        }
    }

    // E^{n+1}; Hy and Hx of plane k-1 from the plane before
    const bool j_int = FAST || (j >= 1 && j <= N - 1);
    const bool k_int = FAST || (k >= 1 && k <= Nk - 1);
    float exn[V], eyn[V], ezn[V];
    if constexpr (FAST && !MAT) {
        // packed pairs; only the i = 0 wall cell (lane 0 of the first
        // block) keeps its Ey and Ez
        float dzi[V], dyi[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            dzi[e] = __fsub_rn(hzn[e], (e > 0) ? hzn[e - 1] : hz_first);
            dyi[e] = __fsub_rn(hyn[e], (e > 0) ? hyn[e - 1] : hy_first);
        }
#pragma unroll
        for (int e = 0; e < V; e += 2) {
            curl2(&ex[e], s, d2(&hzn[e], &hzjmn[e]), d2(&hyn[e], &hykm[e]), &exn[e]);
            curl2(&ey[e], s, d2(&hxn[e], &hxkm[e]), p2(dzi[e], dzi[e + 1]), &eyn[e]);
            curl2(&ez[e], s, p2(dyi[e], dyi[e + 1]), d2(&hxn[e], &hxjmn[e]), &ezn[e]);
        }
        if (i0 == 0) {
            eyn[0] = ey[0];
            ezn[0] = ez[0];
        }
    } else
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = i0 + e;
        const bool i_int = FAST ? (e > 0 || i0 > 0) : (i >= 1 && i <= N - 1);
        const float hz_im = (e > 0) ? hzn[e - 1] : hz_first;
        const float hy_im = (e > 0) ? hyn[e - 1] : hy_first;
        if constexpr (MAT) {
            const float2 m = s_me[id[e]];
            exn[e] = ((FAST || i < N) && j_int && k_int) ? curl_add_m(ex[e], m, hzn[e], hzjmn[e], hyn[e], hykm[e]) : ex[e];
            eyn[e] = ((FAST || j < N) && i_int && k_int) ? curl_add_m(ey[e], m, hxn[e], hxkm[e], hzn[e], hz_im) : ey[e];
            ezn[e] = ((FAST || k < Nk) && i_int && j_int) ? curl_add_m(ez[e], m, hyn[e], hy_im, hxn[e], hxjmn[e]) : ez[e];
        } else {
            exn[e] = ((FAST || i < N) && j_int && k_int) ? curl_add(ex[e], s, hzn[e], hzjmn[e], hyn[e], hykm[e]) : ex[e];
            eyn[e] = ((FAST || j < N) && i_int && k_int) ? curl_add(ey[e], s, hxn[e], hxkm[e], hzn[e], hz_im) : ey[e];
            ezn[e] = ((FAST || k < Nk) && i_int && j_int) ? curl_add(ez[e], s, hyn[e], hy_im, hxn[e], hxjmn[e]) : ez[e];
        }
    }
    float x_ex = 0.f, x_hx = 0.f, x_hy = 0.f, x_hz = 0.f, x_ez = ez_r;
    const bool xcell = ALN && lane == 31 && i0 + V == N;
    if (xcell) {
        x_ex = load_scalar(Ex + o + V);
        x_hx = load_scalar(Hx + o + V);
        x_hy = load_scalar(Hy + o + V);
        x_hz = load_scalar(Hz + o + V);
        if (FAST || (j < N && k < Nk)) {
            if constexpr (MAT) x_hx = curl_sub_m(x_hx, s_mh[load_id(a.mat + o + V)], ezj1_x, ez_r, eyk1_x, ey_r);
            else x_hx = curl_sub(x_hx, s, ezj1_x, ez_r, eyk1_x, ey_r);
        }
    }
    if (j == a.sj && k == a.sk && (FAST || act_i)) {
        const bool in_vec = (a.si >= i0 && a.si < i0 + V);
        const bool in_extra = xcell && a.si == N;
        if (in_vec || in_extra) {
            const long long n = *a.counter;
            if (a.src_on) {
                const float u = __fdiv_rn(__fsub_rn((float)n, a.delay), a.width);
                const float gsrc = __fmul_rn(a.amp, expf(-u * u));
                if (in_vec) {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (i0 + e == a.si) ezn[e] = __fadd_rn(ezn[e], gsrc);
                } else {
                    x_ez = __fadd_rn(x_ez, gsrc);
                }
            }
            *a.counter = n + 1;
        }
    }
    if (FAST || act_i) {
        const int nv = FAST ? V : M - i0;
        store_vecw<ST, V>(static_cast<ST*>(a.g[EX]) + o, exn, nv);
        store_vecw<ST, V>(static_cast<ST*>(a.g[EY]) + o, eyn, nv);
        store_vecw<ST, V>(static_cast<ST*>(a.g[EZ]) + o, ezn, nv);
        store_vecw<ST, V>(static_cast<ST*>(a.g[HX]) + o, hxn, nv);
        store_vecw<ST, V>(static_cast<ST*>(a.g[HY]) + o, hyn, nv);
        store_vecw<ST, V>(static_cast<ST*>(a.g[HZ]) + o, hzn, nv);
        if (xcell) {
            store_scalar(static_cast<ST*>(a.g[EX]) + o + V, x_ex);
            store_scalar(static_cast<ST*>(a.g[EY]) + o + V, ey_r);
            store_scalar(static_cast<ST*>(a.g[EZ]) + o + V, x_ez);
            store_scalar(static_cast<ST*>(a.g[HX]) + o + V, x_hx);
            store_scalar(static_cast<ST*>(a.g[HY]) + o + V, x_hy);
            store_scalar(static_cast<ST*>(a.g[HZ]) + o + V, x_hz);
        }
    }
    // carried to plane k+1
#pragma unroll
    for (int e = 0; e < V; ++e) {
        ex[e] = ex1[e];
        ey[e] = ey1[e];
        ez[e] = ez1[e];
        hykm[e] = hyn[e];
        hxkm[e] = hxn[e];
        eyjm[e] = eyjm1[e];
    }
}

// Planes ahead of the march whose streaming vectors (H at (j, k), E at
// (j, k+1)) a thread asks L2 to fetch from DRAM, so that their loads, a few
// planes later, wait on L2 instead of DRAM.  A prefetch takes no register
// and is issued only for addresses inside the arrays.
constexpr int kMarchPrefetch = 2;

template <typename ST>
__device__ __forceinline__ void march_prefetch_l2(const FdtdArgs& a, long long row_o, int k) {
    const int Mk = a.Nk + 1;
    if (k >= Mk) return;
    const long long o = (long long)k * a.plane + row_o;
    const long long o1 = (k + 1 < Mk) ? o + a.plane : o;
#pragma unroll
    for (int f = HX; f <= HZ; ++f)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(static_cast<const ST*>(a.f[f]) + o)));
#pragma unroll
    for (int f = EX; f <= EZ; ++f)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(static_cast<const ST*>(a.f[f]) + o1)));
}

// A vector load whose lines L2 keeps ahead of normally cached ones (an
// evict_last cache policy): the planes at a chunk's lower edge, which the
// block of the chunk below reads again at the end of its march, one block's
// run later.
template <typename ST, int W>
__device__ __forceinline__ void load_vecw_keep(const ST* p, float (&v)[W], unsigned long long pol) {
    static_assert(W * sizeof(ST) == 8 || W * sizeof(ST) == 16, "8- or 16-byte access");
    if (!GS_CHK(p, W * sizeof(ST))) {
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = 0.f;
        return;
    }
    const size_t g = __cvta_generic_to_global(p);
    if constexpr (W * sizeof(ST) == 16) {
        uint4 raw;
        asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(raw.x), "=r"(raw.y), "=r"(raw.z), "=r"(raw.w)
                     : "l"(g), "l"(pol));
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    } else {
        uint2 raw;
        asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                     : "=r"(raw.x), "=r"(raw.y)
                     : "l"(g), "l"(pol));
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = to_f32(e[i]);
    }
}

template <typename ST, bool ALN, bool MAT>
__global__ void __launch_bounds__(256, 2) fdtd_fused_march_kernel(const FdtdArgs a) {
    constexpr int V = kFdtdColumnCells;
    pdl_wait_then_trigger();
    // media: the H rows (da, db) and the E rows (ca, cb) of the table
    __shared__ float2 s_mh[MAT ? 256 : 1], s_me[MAT ? 256 : 1];
    if constexpr (MAT) {
        const int nt = 32 * blockDim.y;
        for (int t = threadIdx.x + 32 * threadIdx.y; t < 256; t += nt) {
            s_mh[t] = __ldg(a.med + t);
            s_me[t] = __ldg(a.med + 256 + t);
        }
        __syncthreads();
    }
    const int N = a.N, M = N + 1, Nk = a.Nk, Mk = Nk + 1;
    const int lane = threadIdx.x;
    const uint3 blk = block_index(a.rev);
    const int i0 = (blk.x * 32 + lane) * V;
    const int j = blk.y * blockDim.y + threadIdx.y;
    if (j >= M) return;  // the whole warp: j is one per warp (after the block's one barrier)
    const int k0 = blk.z * a.kmarch;
    const int k1 = min(k0 + a.kmarch, Mk);
    const bool act_i = ALN || i0 < M;
    const bool in_x = ALN || __all_sync(0xffffffffu, i0 + V <= N);
    const bool fast_j = in_x && j >= 1 && j <= N - 1;
    const long long P = a.pitch, PL = a.plane;
    const long long dj1 = (j + 1 < M) ? P : 0;
    const long long djm = (j >= 1) ? -P : 0;
    const long long o = (long long)k0 * PL + (long long)j * P + (act_i ? i0 : 0);
    const ST* Ex = static_cast<const ST*>(a.f[EX]);
    const ST* Ey = static_cast<const ST*>(a.f[EY]);
    const ST* Ez = static_cast<const ST*>(a.f[EZ]);
    unsigned long long keep;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
    float ex[V], ey[V], ez[V], eyjm[V], hykm[V], hxkm[V];
    load_vecw_keep<ST, V>(Ex + o, ex, keep);
    load_vecw_keep<ST, V>(Ey + o, ey, keep);
    load_vecw_keep<ST, V>(Ez + o, ez, keep);
    load_vecw_keep<ST, V>(Ey + o + djm, eyjm, keep);
    if (k0 >= 1) {
        // H^{n+1/2} of Hy and Hx on plane k0-1, as its owner computes it
        const ST* Hx = static_cast<const ST*>(a.f[HX]);
        const ST* Hy = static_cast<const ST*>(a.f[HY]);
        const float s = a.s;
        float hyo[V], hxo[V], exkm[V], ezkm[V], eykm[V], ezj1km[V];
        load_vecw_keep<ST, V>(Hy + o - PL, hyo, keep);
        load_vecw_keep<ST, V>(Hx + o - PL, hxo, keep);
        load_vecw_keep<ST, V>(Ex + o - PL, exkm, keep);
        load_vecw_keep<ST, V>(Ez + o - PL, ezkm, keep);
        load_vecw_keep<ST, V>(Ey + o - PL, eykm, keep);
        load_vecw_keep<ST, V>(Ez + o - PL + dj1, ezj1km, keep);
        const bool has_r = (lane == 31) && act_i && (i0 + V < M);
        const float ezkm_r = has_r ? load_scalar(Ez + o - PL + V) : 0.f;
        const float ezkm_n = __shfl_down_sync(0xffffffffu, ezkm[0], 1);
        const float ezkm_last = (lane == 31) ? ezkm_r : ezkm_n;
        unsigned idkm[V];
        if constexpr (MAT) load_ids<V>(a.mat + o - PL, idkm);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const float ezkm_ip = (e + 1 < V) ? ezkm[e + 1] : ezkm_last;
            if constexpr (MAT) {
                const float2 m = s_mh[idkm[e]];
                hykm[e] = stored<ST>((i0 + e < N) ? curl_sub_m(hyo[e], m, ex[e], exkm[e], ezkm_ip, ezkm[e]) : hyo[e]);
                hxkm[e] = stored<ST>((j < N) ? curl_sub_m(hxo[e], m, ezj1km[e], ezkm[e], ey[e], eykm[e]) : hxo[e]);
            } else {
                hykm[e] = stored<ST>((i0 + e < N) ? curl_sub(hyo[e], s, ex[e], exkm[e], ezkm_ip, ezkm[e]) : hyo[e]);
                hxkm[e] = stored<ST>((j < N) ? curl_sub(hxo[e], s, ezj1km[e], ezkm[e], ey[e], eykm[e]) : hxo[e]);
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) hykm[e] = hxkm[e] = 0.f;  // k = 0 is a wall: not read
    }
    const long long row_o = (long long)j * P + (act_i ? i0 : 0);
#pragma unroll
    for (int d = 1; d < kMarchPrefetch; ++d)
        if (k0 + d < k1) march_prefetch_l2<ST>(a, row_o, k0 + d);
    for (int k = k0; k < k1; ++k) {
        if (k + kMarchPrefetch < k1) march_prefetch_l2<ST>(a, row_o, k + kMarchPrefetch);
        if (fast_j && k >= 1 && k <= Nk - 1)
            fdtd_march_plane<ST, true, ALN, MAT>(a, s_mh, s_me, lane, i0, act_i, j, k, ex, ey, ez, hykm, hxkm, eyjm);
        else
            fdtd_march_plane<ST, false, ALN, MAT>(a, s_mh, s_me, lane, i0, act_i, j, k, ex, ey, ez, hykm, hxkm, eyjm);
    }
}

namespace {

template <typename ST>
const void* fdtd_march_func(bool aln, bool mat) {
    if (mat) return aln ? (const void*)fdtd_fused_march_kernel<ST, true, true> : (const void*)fdtd_fused_march_kernel<ST, false, true>;
    return aln ? (const void*)fdtd_fused_march_kernel<ST, true, false> : (const void*)fdtd_fused_march_kernel<ST, false, false>;
}

template <typename ST, bool MAT>
const void* fdtd_column_func(bool e_half, bool aln) {
    if (aln) return e_half ? (const void*)fdtd_e_column_kernel<ST, MAT, true> : (const void*)fdtd_h_column_kernel<ST, MAT, true>;
    return e_half ? (const void*)fdtd_e_column_kernel<ST, MAT, false> : (const void*)fdtd_h_column_kernel<ST, MAT, false>;
}

template <typename ST>
const void* fdtd_func(bool e_half, bool col, bool mat, bool aln) {
    if (!col) return e_half ? (const void*)fdtd_e_kernel<ST> : (const void*)fdtd_h_kernel<ST>;
    return mat ? fdtd_column_func<ST, true>(e_half, aln) : fdtd_column_func<ST, false>(e_half, aln);
}

}  // namespace

cudaError_t fdtd_desc(gs_dtype dt, bool e_half, const FdtdArgs& a, int block_x, int variant, LaunchDesc* out) {
    if (variant == GS_KERNEL_FUSED) {
        const bool aln = (a.N % (32 * kFdtdColumnCells) == 0);
        if (a.mat && a.kmarch < 1) return cudaErrorNotSupported;  // media: the march or the two launches
        if (a.kmarch > 0) {
            // block (32, rows): one warp a row j, marching kmarch planes
            const bool mat = (a.mat != nullptr);
            switch (dt) {
                case GS_F32: out->func = fdtd_march_func<float>(aln, mat); break;
                case GS_BF16: out->func = fdtd_march_func<__nv_bfloat16>(aln, mat); break;
                case GS_F16: out->func = fdtd_march_func<__half>(aln, mat); break;
                default: return cudaErrorInvalidValue;
            }
            const int by = std::max(1, std::min(a.kc, 8));
            const int M = a.N + 1, Mk = a.Nk + 1;
            const int span = aln ? a.N : M;
            out->block = dim3(32, by, 1);
            out->grid = dim3((span + 32 * kFdtdColumnCells - 1) / (32 * kFdtdColumnCells), (M + by - 1) / by,
                             (Mk + a.kmarch - 1) / a.kmarch);
            out->smem = 0;
            out->set_args(a);
            return cudaSuccess;
        }
        switch (dt) {
            case GS_F32: out->func = aln ? (const void*)fdtd_fused_kernel<float, true> : (const void*)fdtd_fused_kernel<float, false>; break;
            case GS_BF16: out->func = aln ? (const void*)fdtd_fused_kernel<__nv_bfloat16, true> : (const void*)fdtd_fused_kernel<__nv_bfloat16, false>; break;
            case GS_F16: out->func = aln ? (const void*)fdtd_fused_kernel<__half, true> : (const void*)fdtd_fused_kernel<__half, false>; break;
            default: return cudaErrorInvalidValue;
        }
        const int by = std::max(1, std::min(a.kc, 8));
        const int bz = std::max(1, 8 / by);
        const int M = a.N + 1, Mk = a.Nk + 1;
        const int span = aln ? a.N : M;
        out->block = dim3(32, by, bz);
        out->grid = dim3((span + 32 * kFdtdColumnCells - 1) / (32 * kFdtdColumnCells), (M + by - 1) / by, (Mk + bz - 1) / bz);
        out->smem = 0;
        out->set_args(a);
        return cudaSuccess;
    }
    const bool col = (variant == GS_KERNEL_COLUMN);
    const int V = col ? kFdtdColumnCells : ((dt == GS_F32) ? 4 : 8);
    const int M = a.N + 1, Mk = a.Nk + 1;
    const bool mat = (a.mat != nullptr);
    if (mat && !col) return cudaErrorNotSupported;  // media: column kernels only
    // ALN: the warps tile i in [0, N) exactly; lane 31 takes the i = N column
    const bool aln = col && (a.N % (32 * V) == 0);
    switch (dt) {
        case GS_F32: out->func = fdtd_func<float>(e_half, col, mat, aln); break;
        case GS_BF16: out->func = fdtd_func<__nv_bfloat16>(e_half, col, mat, aln); break;
        case GS_F16: out->func = fdtd_func<__half>(e_half, col, mat, aln); break;
        default: return cudaErrorInvalidValue;
    }
    if (col) {
        // block (32, by, bz): a.kc rows of j per block (<= 8), 256/(32*by) planes of k
        const int by = std::max(1, std::min(a.kc, 8));
        const int bz = std::max(1, 8 / by);
        out->block = dim3(32, by, bz);
        const int span = aln ? a.N : M;
        out->grid = dim3((span + 32 * V - 1) / (32 * V), (M + by - 1) / by, (Mk + bz - 1) / bz);
    } else {
        const int by = std::max(1, 256 / block_x);
        out->block = dim3(block_x, by, 1);
        out->grid = dim3((M + block_x * V - 1) / (block_x * V), (M + by - 1) / by, (Mk + a.kc - 1) / a.kc);
    }
    out->smem = 0;
    out->set_args(a);
    return cudaSuccess;
}

GS_CHECK_UNIT(fdtd)

}  // namespace gs
