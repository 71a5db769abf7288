// Thermal stencil kernels: 2D 5-point and 3D 7-point explicit updates (the
// roles of Rodinia Hotspot / Hotspot3D in the paper's Sec. III-C), one step
// per launch (depth 1: COLUMN, COLUMN_SMEM, MARCH) or t steps per launch
// (temporal blocking, depth 2 or 4: COLUMN in 2D and WAVE with the levels in
// registers, TILE on an overlapped shared-memory tile), and the persistent
// kernel of an instance batch.
//
// Update (per cell, FP32):
//   T' = T + k*(P + cy*(N+S-2T) + cx*(E+W-2T) + cz*(t_amb-T) [+ cz2*(U+D-2T)])
// Every kernel evaluates it through heat_cell(), whose operations are spelled
// with explicit round-to-nearest intrinsics (no contraction or reassociation
// is possible), so depth-1, temporally blocked, per-step and graph runs are
// bit-identical.
#include <algorithm>

#include <cuda.h>  // CUtensorMap (the tensor map of the STREAM kernel's copies)

#define GS_CHECK_THIS_UNIT  // checked builds bounds-check this unit's field accesses
#include "common.cuh"

namespace gs {

template <bool IS3D>
__device__ __forceinline__ float heat_cell(float t, float n, float s, float w, float e, float d, float u, float p,
                                           const HeatCoef& c) {
    float acc = p;
    acc = __fmaf_rn(c.cy, __fmaf_rn(-2.0f, t, __fadd_rn(n, s)), acc);
    acc = __fmaf_rn(c.cx, __fmaf_rn(-2.0f, t, __fadd_rn(w, e)), acc);
    acc = __fmaf_rn(c.cz, __fsub_rn(c.t_amb, t), acc);
    if (IS3D) acc = __fmaf_rn(c.cz2, __fmaf_rn(-2.0f, t, __fadd_rn(d, u)), acc);
    return __fmaf_rn(c.k, acc, t);
}

// A level computed inside a temporally blocked launch, rounded to the
// storage type exactly as a depth-1 launch's store rounds it (identity for
// f32), so that a depth-t launch equals t depth-1 launches in every storage
// type.
template <typename ST>
__device__ __forceinline__ float as_stored(float v) {
    return to_f32(from_f32<ST>(v));
}

// heat_cell for two adjacent cells with Blackwell's packed FP32 pair
// operations (add/sub/fma .rn.f32x2): each half is rounded exactly as the
// scalar operation of heat_cell, in the same order, so the results are the
// same bits.  The x-neighbour sums w+e arrive already rounded (scalar adds:
// the shifted neighbours are not register pairs).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <bool IS3D>
__device__ __forceinline__ void heat_cell_x2(const float* t, const float* n, const float* s, const float* xs,
                                             const float* d, const float* u, const float* p, const HeatCoef& c,
                                             float* out) {
    const unsigned long long T = f2_pack(t[0], t[1]);
    const unsigned long long M2 = f2_pack(-2.0f, -2.0f);
    unsigned long long acc = f2_pack(p[0], p[1]);
    acc = f2_fma(f2_pack(c.cy, c.cy), f2_fma(M2, T, f2_add(f2_pack(n[0], n[1]), f2_pack(s[0], s[1]))), acc);
    acc = f2_fma(f2_pack(c.cx, c.cx), f2_fma(M2, T, f2_pack(xs[0], xs[1])), acc);
    acc = f2_fma(f2_pack(c.cz, c.cz), f2_sub(f2_pack(c.t_amb, c.t_amb), T), acc);
    if (IS3D) acc = f2_fma(f2_pack(c.cz2, c.cz2), f2_fma(M2, T, f2_add(f2_pack(d[0], d[1]), f2_pack(u[0], u[1]))), acc);
    f2_unpack(f2_fma(f2_pack(c.k, c.k), acc, T), out[0], out[1]);
}

// heat_cell_x2 (3D) with the z-neighbour sums d+u already formed (scalar
// round-to-nearest adds, as the packed add rounds each half): for a plane
// pair the planes below and above are no aligned register pair.
__device__ __forceinline__ void heat_cell_x2z(const float* t, const float* n, const float* s, const float* xs,
                                              const float* zs, const float* p, const HeatCoef& c, float* out) {
    const unsigned long long T = f2_pack(t[0], t[1]);
    const unsigned long long M2 = f2_pack(-2.0f, -2.0f);
    unsigned long long acc = f2_pack(p[0], p[1]);
    acc = f2_fma(f2_pack(c.cy, c.cy), f2_fma(M2, T, f2_add(f2_pack(n[0], n[1]), f2_pack(s[0], s[1]))), acc);
    acc = f2_fma(f2_pack(c.cx, c.cx), f2_fma(M2, T, f2_pack(xs[0], xs[1])), acc);
    acc = f2_fma(f2_pack(c.cz, c.cz), f2_sub(f2_pack(c.t_amb, c.t_amb), T), acc);
    acc = f2_fma(f2_pack(c.cz2, c.cz2), f2_fma(M2, T, f2_pack(zs[0], zs[1])), acc);
    f2_unpack(f2_fma(f2_pack(c.k, c.k), acc, T), out[0], out[1]);
}

// 16-byte shared-memory row segments (V is 4 or 8 floats).
template <int V>
__device__ __forceinline__ void sm_put(float* p, const float (&v)[V]) {
#pragma unroll
    for (int i = 0; i < V; i += 4) *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}
template <int V>
__device__ __forceinline__ void sm_get(const float* p, float (&v)[V]) {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
        const float4 q = *reinterpret_cast<const float4*>(p + i);
        v[i] = q.x; v[i + 1] = q.y; v[i + 2] = q.z; v[i + 3] = q.w;
    }
}

// Value a missing neighbour reads: the cell itself (clamp) or 0 (Dirichlet-0).
template <int BC>
__device__ __forceinline__ float bnd(float self) {
    return BC == GS_BC_CLAMP ? self : 0.0f;
}

// ------------------------------------------------------------ depth 1 ----
//
// Block = blockDim.x threads along x (each owning one 16-byte vector of V
// cells) x blockDim.y z-planes (3D).  The block marches `rows` rows in y;
// each thread keeps rows y-1, y, y+1 of its vector in registers and issues
// the loads of row y+2 (and P, edge scalars, z-halo rows of row y+1) one
// iteration ahead.  x-neighbours come from warp shuffles (lanes 0/31 load
// one scalar each); z-neighbours come from a double-buffered shared-memory
// row per plane.
// One block's share of a depth-1 step: the tile (bx, by[, bz]) of the grid
// described by `a`.  Shared by the single-grid kernel and the persistent
// multi-instance kernel.
//
// The row window (rows y-1, y, y+1 and the prefetch target y+2) is a ring of
// four register arrays rotated by a 4-way manual unroll, so the march moves
// no data between registers.  z-boundaries need no per-cell select: the
// thread on the bottom (top) plane writes the boundary value of its own row
// into the shared row below (above) it, and threads past nz write nothing.
// x-boundaries are handled per cell only in warps that touch the grid's x
// edges; interior warps take a select-free path (a warp-uniform branch with
// no barrier inside).  Planes without a source keep P at zero.
template <typename ST, int BC, bool IS3D>
struct MarchTile {
    static constexpr int V = Vec<ST>::N;
    const HeatArgs& a;
    const ST* col;   // this thread's vector in row 0 of its plane
    const ST* pcol;  // P, row 0
    const ST* dcol;  // plane z0-1 (tz == 0 halo)
    const ST* ucol;  // plane z0+ZB (tz == ZB-1 halo)
    ST* ocol;        // output, row 0 of this plane
    float* zsm;
    int lane, tx, tz, ZB, z, x0, nx, ny, y1, rowlen;
    bool act, has_p, dn_halo, up_halo, fast_x;

    __device__ __forceinline__ void fill_bnd(float (&dst)[V], const float (&src)[V]) const {
#pragma unroll
        for (int i = 0; i < V; ++i) dst[i] = bnd<BC>(src[i]);
    }

    // One output row y.  prv/cur/nxt hold rows y-1, y, y+1 (boundary rows
    // materialised); nn receives row y+2; pc/dc/uc/wl/er are row y's P,
    // z-halos and x-edge scalars, pn/dn/un/wln/ern receive row y+1's.
    __device__ __forceinline__ void step(int y, float (&prv)[V], float (&cur)[V], float (&nxt)[V], float (&nn)[V],
                                         float (&pc)[V], float (&pn)[V], float (&dc)[V], float (&dn)[V],
                                         float (&uc)[V], float (&un)[V], float& wl, float& wln, float& er,
                                         float& ern) const {
        const bool more = (y + 1 < y1);
        const long long pitch = a.pitch;
#pragma unroll
        for (int i = 0; i < V; ++i) { pn[i] = 0.f; dn[i] = 0.f; un[i] = 0.f; }
        wln = 0.f;
        ern = 0.f;
        if (act && more && y + 2 < ny) load_vec(col + (long long)(y + 2) * pitch, nn);
        if (act && more && has_p) load_vec(pcol + (long long)(y + 1) * a.p_pitch, pn);
        if (act && more && lane == 0 && x0 > 0) wln = load_scalar(col + (long long)(y + 1) * pitch - 1);
        if (act && more && lane == 31 && x0 + V < nx) ern = load_scalar(col + (long long)(y + 1) * pitch + V);
        if (dn_halo && more) load_vec(dcol + (long long)(y + 1) * pitch, dn);
        if (up_halo && more) load_vec(ucol + (long long)(y + 1) * pitch, un);

        float w0 = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
        float eV = __shfl_down_sync(0xffffffffu, cur[0], 1);
        if (lane == 0) w0 = wl;
        if (lane == 31) eV = er;

        float dv[V], uv[V];
        if (IS3D) {
            float* buf = zsm + (size_t)(y & 1) * (ZB + 2) * rowlen + tx * V;
            if (z < a.nz) sm_put<V>(buf + (tz + 1) * rowlen, cur);
            if (dn_halo) sm_put<V>(buf, dc);
            if (tz == ZB - 1 && up_halo) sm_put<V>(buf + (ZB + 1) * rowlen, uc);
            if (z == 0 || z + 1 == a.nz) {
                float b[V];
                fill_bnd(b, cur);
                if (z == 0) sm_put<V>(buf + tz * rowlen, b);
                if (z + 1 == a.nz) sm_put<V>(buf + (tz + 2) * rowlen, b);
            }
            __syncthreads();
            sm_get<V>(buf + tz * rowlen, dv);
            sm_get<V>(buf + (tz + 2) * rowlen, uv);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) { dv[i] = 0.f; uv[i] = 0.f; }
        }

        if (act) {
            float out[V];
            if (fast_x) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const float w = (i == 0) ? w0 : cur[i - 1];
                    const float e = (i == V - 1) ? eV : cur[i + 1];
                    out[i] = heat_cell<IS3D>(cur[i], prv[i], nxt[i], w, e, dv[i], uv[i], pc[i], a.c);
                }
                store_vec(ocol + (long long)y * pitch, out, V);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const int x = x0 + i;
                    const float t = cur[i];
                    float w = (i == 0) ? w0 : cur[i - 1];
                    float e = (i == V - 1) ? eV : cur[i + 1];
                    if (x == 0) w = bnd<BC>(t);
                    if (x + 1 >= nx) e = bnd<BC>(t);
                    out[i] = heat_cell<IS3D>(t, prv[i], nxt[i], w, e, dv[i], uv[i], pc[i], a.c);
                }
                store_vec(ocol + (long long)y * pitch, out, nx - x0);
            }
        }
        // the row after nxt is nn; past the last row it is the boundary row
        if (y + 2 >= ny) fill_bnd(nn, nxt);
    }

};

template <typename ST, int BC, bool IS3D>
__device__ __forceinline__ void heat_march_tile(const HeatArgs& a, int bx, int by, int bz, float* zsm) {
    constexpr int V = Vec<ST>::N;
    const int BX = blockDim.x;
    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int x0 = (bx * BX + tx) * V;
    const int nx = a.nx, ny = a.ny;
    const int ZB = IS3D ? (int)blockDim.y : 1;
    const int tz = IS3D ? (int)threadIdx.y : 0;
    const int z0 = IS3D ? bz * ZB : 0;
    const int z = z0 + tz;
    const int y0 = by * a.rows;
    const int y1 = min(y0 + a.rows, ny);
    const long long zoff = IS3D ? (long long)z * a.plane : 0;
    const ST* Tin = static_cast<const ST*>(a.Tin);

    MarchTile<ST, BC, IS3D> m{a};
    m.col = Tin + zoff + x0;
    m.pcol = static_cast<const ST*>(a.P) + x0;
    m.dcol = Tin + zoff - a.plane + x0;
    m.ucol = Tin + zoff + a.plane + x0;
    m.ocol = static_cast<ST*>(a.Tout) + zoff + x0;
    m.zsm = zsm;
    m.lane = lane;
    m.tx = tx;
    m.tz = tz;
    m.ZB = ZB;
    m.z = z;
    m.x0 = x0;
    m.nx = nx;
    m.ny = ny;
    m.y1 = y1;
    m.rowlen = BX * V;
    m.act = (x0 < nx) && (!IS3D || z < a.nz);
    m.has_p = !IS3D || z == 0;
    m.dn_halo = IS3D && tz == 0 && z0 > 0 && x0 < nx;
    m.up_halo = IS3D && tz == ZB - 1 && z0 + ZB < a.nz && x0 < nx;
    m.fast_x = __all_sync(0xffffffffu, x0 > 0 && x0 + V < nx);

    float A[V], B[V], C[V], D[V], PA[V], PB[V], DA[V], DB[V], UA[V], UB[V];
    float WA = 0.f, WB = 0.f, EA = 0.f, EB = 0.f;
#pragma unroll
    for (int i = 0; i < V; ++i) { B[i] = 0.f; D[i] = 0.f; PA[i] = 0.f; DA[i] = 0.f; UA[i] = 0.f; }
    // Prologue: A = row y0-1, B = row y0, C = row y0+1 (boundary rows
    // materialised) and row y0's P, z-halos and x-edge scalars.
    const long long pitch = a.pitch;
    if (m.act) load_vec(m.col + (long long)y0 * pitch, B);
    if (m.act && y0 > 0) load_vec(m.col + (long long)(y0 - 1) * pitch, A);
    else m.fill_bnd(A, B);
    if (m.act && y0 + 1 < ny) load_vec(m.col + (long long)(y0 + 1) * pitch, C);
    else m.fill_bnd(C, B);
    if (m.act && m.has_p) load_vec(m.pcol + (long long)y0 * a.p_pitch, PA);
    if (m.act && lane == 0 && x0 > 0) WA = load_scalar(m.col + (long long)y0 * pitch - 1);
    if (m.act && lane == 31 && x0 + V < nx) EA = load_scalar(m.col + (long long)y0 * pitch + V);
    if (m.dn_halo) load_vec(m.dcol + (long long)y0 * pitch, DA);
    if (m.up_halo) load_vec(m.ucol + (long long)y0 * pitch, UA);

    for (int y = y0; y < y1;) {
        m.step(y, A, B, C, D, PA, PB, DA, DB, UA, UB, WA, WB, EA, EB);
        if (++y >= y1) break;
        m.step(y, B, C, D, A, PB, PA, DB, DA, UB, UA, WB, WA, EB, EA);
        if (++y >= y1) break;
        m.step(y, C, D, A, B, PA, PB, DA, DB, UA, UB, WA, WB, EA, EB);
        if (++y >= y1) break;
        m.step(y, D, A, B, C, PB, PA, DB, DA, UB, UA, WB, WA, EB, EA);
        ++y;
    }
}

template <typename ST, int BC, bool IS3D>
__global__ void __launch_bounds__(512) heat_step_kernel(const HeatArgs a) {
    extern __shared__ float zsm[];  // [2][ZB+2][BX*V] (3D only)
    pdl_wait_then_trigger();
    const uint3 b = block_index(a.rev);
    heat_march_tile<ST, BC, IS3D>(a, b.x, b.y, b.z, zsm);
}

template <typename ST, int BC, int NZM, int W = Vec<ST>::N>
__device__ __forceinline__ void heat_column_tile(const HeatArgs& a, int bx, int by);
template <typename ST, int BC, int T, int R>
__device__ __forceinline__ void heat_column_t_tile(const HeatArgs& a, int bx, int by);

// Output rows per thread of the depth-T column kernel (register budget).
template <typename ST>
__host__ __device__ constexpr int column_t_rows() {
    return Vec<ST>::N == 4 ? 4 : 2;
}

// ------------------------------------------------- multi-instance (2D) ----
//
// Persistent kernel over many independent 2D grids: the work list is every
// (instance, x tile, y tile) of the depth-1 march, instances ordered largest
// first; block b takes items b, b + gridDim.x, ...  The descriptor table
// (per instance: both buffers, P, sizes, pitches, first work item) lives in
// device memory; `parity` selects which buffer is read.
// KIND: 0 MARCH tiles (blockDim.x threads marching `rows` rows), 1 COLUMN
// tiles (32 x blockDim.y threads, one row per warp row), 2 or 4: COLUMN
// tiles of that temporal depth (30 stored vectors x column_t_rows() rows per
// warp row; the launch advances every instance that many steps).
template <typename ST, int BC, int KIND>
__global__ void __launch_bounds__(512) heat_multi_kernel(const MultiArgs m) {
    pdl_wait_then_trigger();
    const int V = Vec<ST>::N;
    const int span = (KIND == 0 ? (int)blockDim.x * V : KIND == 1 ? 32 * V : 30 * V);
    for (int w0 = blockIdx.x; w0 < m.total_items; w0 += gridDim.x) {
        const int w = m.rev ? m.total_items - 1 - w0 : w0;
        // binary search: last instance whose first item <= w
        int lo = 0, hi = m.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (m.desc[mid].first_item <= w) lo = mid;
            else hi = mid - 1;
        }
        const MultiInstance& d = m.desc[lo];
        HeatArgs a{};
        a.Tin = m.parity ? d.T1 : d.T0;
        a.Tout = m.parity ? d.T0 : d.T1;
        a.P = d.P;
        a.nx = d.nx;
        a.ny = d.ny;
        a.nz = 1;
        a.rows = m.rows;
        a.pitch = d.pitch;
        a.plane = d.pitch * d.ny;
        a.p_pitch = d.p_pitch;
        a.c = m.c;
        const int ntx = (d.nx + span - 1) / span;
        const int item = w - d.first_item;
        if constexpr (KIND == 0) heat_march_tile<ST, BC, false>(a, item % ntx, item / ntx, 0, nullptr);
        else if constexpr (KIND == 1) heat_column_tile<ST, BC, 1>(a, item % ntx, item / ntx);
        else heat_column_t_tile<ST, BC, KIND, column_t_rows<ST>()>(a, item % ntx, item / ntx);
    }
}

// ----------------------------------------------------- temporal blocking --
//
// One block owns an output tile of tile_x x tile_y columns (all nz layers).
// It loads the tile plus a halo of width D into shared memory, advances D
// steps there (the valid region shrinks by one cell per side per step), and
// writes the tile interior.  Cells outside the grid are never read by valid
// cells: boundary neighbours are selected by global coordinates exactly as
// in the depth-1 kernel, and the same heat_cell() does the arithmetic, so
// one depth-D launch equals D depth-1 launches bit for bit.
//
// Shared memory: two buffers of nz*(tile_y+2D)*(tile_x+2D) floats plus the
// P tile of (tile_y+2D)*(tile_x+2D) floats.
template <typename ST, int BC, bool IS3D, int D>
__global__ void __launch_bounds__(512) heat_temporal_kernel(const HeatArgs a) {
    extern __shared__ float tsm[];
    pdl_wait_then_trigger();

    const int IX = a.tile_x + 2 * D;
    const int IY = a.tile_y + 2 * D;
    const int nz = IS3D ? a.nz : 1;
    const int area = IX * IY;
    const int vol = area * nz;
    float* bufA = tsm;
    float* bufB = tsm + vol;
    float* ptile = tsm + 2 * vol;
    const uint3 blk = block_index(a.rev);
    const int gx0 = blk.x * a.tile_x - D;  // global x of local ix = 0
    const int gy0 = blk.y * a.tile_y - D;
    const int nx = a.nx, ny = a.ny;
    const ST* __restrict__ Tin = static_cast<const ST*>(a.Tin);
    ST* __restrict__ Tout = static_cast<ST*>(a.Tout);
    const ST* __restrict__ P = static_cast<const ST*>(a.P);
    const int nthr = blockDim.x;

    // Load the input region (cells outside the grid are left as 0).
    for (int idx = threadIdx.x; idx < vol; idx += nthr) {
        const int ix = idx % IX;
        const int iy = (idx / IX) % IY;
        const int iz = idx / area;
        const int gx = gx0 + ix, gy = gy0 + iy;
        float v = 0.f;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny)
            v = load_scalar(Tin + (long long)iz * a.plane + (long long)gy * a.pitch + gx);
        bufA[idx] = v;
    }
    for (int idx = threadIdx.x; idx < area; idx += nthr) {
        const int ix = idx % IX;
        const int iy = idx / IX;
        const int gx = gx0 + ix, gy = gy0 + iy;
        float v = 0.f;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) v = load_scalar(P + (long long)gy * a.p_pitch + gx);
        ptile[idx] = v;
    }
    __syncthreads();

#pragma unroll 1
    for (int s = 1; s <= D; ++s) {
        const int wx = IX - 2 * s, wy = IY - 2 * s;
        const int warea = wx * wy;
        const int wvol = warea * nz;
        for (int idx = threadIdx.x; idx < wvol; idx += nthr) {
            const int ix = s + idx % wx;
            const int iy = s + (idx / wx) % wy;
            const int iz = idx / warea;
            const int gx = gx0 + ix, gy = gy0 + iy;
            if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
            const int l = iz * area + iy * IX + ix;
            const float t = bufA[l];
            const float w = (gx > 0) ? bufA[l - 1] : bnd<BC>(t);
            const float e = (gx + 1 < nx) ? bufA[l + 1] : bnd<BC>(t);
            const float n = (gy > 0) ? bufA[l - IX] : bnd<BC>(t);
            const float so = (gy + 1 < ny) ? bufA[l + IX] : bnd<BC>(t);
            float d = 0.f, u = 0.f;
            if (IS3D) {
                d = (iz > 0) ? bufA[l - area] : bnd<BC>(t);
                u = (iz + 1 < nz) ? bufA[l + area] : bnd<BC>(t);
            }
            const float p = (!IS3D || iz == 0) ? ptile[iy * IX + ix] : 0.0f;
            bufB[l] = as_stored<ST>(heat_cell<IS3D>(t, n, so, w, e, d, u, p, a.c));
        }
        __syncthreads();
        float* sw = bufA;
        bufA = bufB;
        bufB = sw;
    }

    // Store the tile interior.
    const int ovol = a.tile_x * a.tile_y * nz;
    for (int idx = threadIdx.x; idx < ovol; idx += nthr) {
        const int ox = idx % a.tile_x;
        const int oy = (idx / a.tile_x) % a.tile_y;
        const int iz = idx / (a.tile_x * a.tile_y);
        const int gx = gx0 + D + ox, gy = gy0 + D + oy;
        if (gx >= nx || gy >= ny) continue;
        const float v = bufA[iz * area + (oy + D) * IX + (ox + D)];
        store_scalar(Tout + (long long)iz * a.plane + (long long)gy * a.pitch + gx, v);
    }
}

// Cells per thread of the COLUMN kernel: a full 16-byte vector in 2D; in 3D
// (every plane of the column in registers) four cells, a 16-byte f32 or an
// 8-byte bf16/f16 access, which keeps the three register arrays of a column
// of eight planes within the 128 registers that two blocks of 256 threads
// per SM leave each thread.
template <typename ST>
constexpr int column_width(bool is3d) {
    return is3d ? 4 : Vec<ST>::N;
}

// --------------------------------------------------------------- column --
//
// Depth 1 without a march: each thread owns W cells along x at one y and
// keeps every plane of its column (nz <= NZM) in registers, so one round of
// independent loads (the P row, then rows y-1, y, y+1 of every plane and the
// x-edge scalars of lanes 0 and 31) feeds the whole update.  x-neighbours
// come from warp shuffles, y- and z-neighbours from registers; no shared
// memory and no barrier.  Vertical reuse between the rows of a block goes
// through L1 (read-only path).  Block (32, rows).
//
// Every load uses coordinates clamped into the grid, so every thread reads
// valid memory (threads past the grid's edge only skip their stores) and no
// register needs a zero fill.  Under the clamp boundary the clamped address
// IS the boundary value (a missing neighbour reads the cell itself), so the
// update needs no per-cell select, except at a ragged row end (a partial
// last vector).  The Dirichlet-0 boundary selects zeros by coordinate.
// EXACT (nz == NZM) makes every z-boundary a compile-time choice.  FAST is
// the warp-uniform common case (every vector of the warp inside the row, the
// warp's row inside the grid): no per-cell edge checks, full-vector stores.
// The kernel is latency- and issue-bound when L2-resident, so instruction
// count and load order matter: the P row first (measured 9-12 % faster in
// 2D), one predicated edge load per plane serving both lanes 0 and 31.
template <typename ST, int BC, int NZM, int W, bool EXACT, bool FAST, bool DEEP>
__device__ __forceinline__ void heat_column_body(const HeatArgs& a, int x0, int y, int z0, bool full_x,
                                                 bool inner_x) {
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    // planes this thread updates: z0 .. z0 + nz - 1 (DEEP: one chunk of a
    // deeper stack, else the whole stack from z0 = 0)
    const int nz = EXACT ? NZM : (DEEP ? min(NZM, a.nz - z0) : a.nz);
    const bool act = FAST || ((x0 < nx) && (y < ny));
    const long long pitch = a.pitch, plane = a.plane;
    const int xc = FAST ? x0 : min(x0, (nx - 1) / W * W);  // last vector's start when past the row
    const int yc = FAST ? y : min(y, ny - 1);
    const long long dn = (yc > 0) ? -pitch : 0;       // row above, clamped
    const long long ds = (yc + 1 < ny) ? pitch : 0;   // row below, clamped
    // lane 0 reads its west scalar, lane 31 its east scalar, both clamped
    const int dedge = (lane == 0) ? ((xc > 0) ? -1 : 0) : min(W, nx - 1 - xc);
    const ST* __restrict__ rc = static_cast<const ST*>(a.Tin) + (long long)yc * pitch + xc;

    float c[NZM][W], n[NZM][W], so[NZM][W], p[W], edge[NZM];
    load_vecw<ST, W>(static_cast<const ST*>(a.P) + (long long)yc * a.p_pitch + xc, p);
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
        // planes past nz (general kernel only) re-read the last plane and
        // are never updated: a branch-free load keeps the register arrays
        // from spilling
        const ST* q = rc + (long long)(z0 + (EXACT ? z : min(z, nz - 1))) * plane;
        load_vecw<ST, W>(q, c[z]);
        load_vecw<ST, W>(q + dn, n[z]);
        load_vecw<ST, W>(q + ds, so[z]);
        edge[z] = 0.f;
        if (lane == 0 || lane == 31) edge[z] = load_scalar(q + dedge);
    }
    // DEEP: the planes just below and above the chunk, at clamped plane
    // indices (at the stack's bottom / top that is the chunk's own edge
    // plane: the clamp boundary's value)
    float cd[W], cu[W];
    if constexpr (DEEP) {
        load_vecw<ST, W>(rc + (long long)max(z0 - 1, 0) * plane, cd);
        load_vecw<ST, W>(rc + (long long)min(z0 + nz, a.nz - 1) * plane, cu);
    }

    ST* out_row = static_cast<ST*>(a.Tout) + (long long)y * pitch + x0;
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
        if (!EXACT && z >= nz) break;  // warp-uniform
        float w0 = __shfl_up_sync(0xffffffffu, c[z][W - 1], 1);
        float eW = __shfl_down_sync(0xffffffffu, c[z][0], 1);
        if (lane == 0) w0 = edge[z];
        if (lane == 31) eW = edge[z];
        if (!act) continue;
        float out[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const float t = c[z][i];
            float w = (i == 0) ? w0 : c[z][i - 1];
            float e = (i == W - 1) ? eW : c[z][i + 1];
            float nv = n[z][i], sv = so[z][i];
            float d = 0.f, u = 0.f;
            if (NZM > 1) {
                const float below = DEEP ? cd[i] : bnd<BC>(t);
                const float above = DEEP ? cu[i] : bnd<BC>(t);
                d = (z > 0) ? c[z > 0 ? z - 1 : 0][i] : below;
                u = (z + 1 < NZM) ? c[z + 1 < NZM ? z + 1 : z][i] : above;
                if (!EXACT) u = (z + 1 < nz) ? u : above;
                if (DEEP && BC == GS_BC_DIRICHLET0) {
                    if (z0 + z == 0) d = 0.f;
                    if (z0 + z + 1 >= a.nz) u = 0.f;
                }
            }
            if (BC == GS_BC_CLAMP) {
                if (!FAST && !full_x && x0 + i + 1 >= nx) e = t;
            } else {
                if (!inner_x) {
                    if (x0 + i == 0) w = 0.f;
                    if (x0 + i + 1 >= nx) e = 0.f;
                }
                if (y == 0) nv = 0.f;
                if (y + 1 >= ny) sv = 0.f;
            }
            out[i] = heat_cell<(NZM > 1)>(t, nv, sv, w, e, d, u, (z == 0 && (!DEEP || z0 == 0)) ? p[i] : 0.0f, a.c);
        }
        store_vecw<ST, W>(out_row + (long long)(z0 + z) * plane, out, (FAST || full_x) ? W : nx - x0);
    }
}

// The COLUMN tile (bx, by): the FAST body for full warps inside the grid,
// the general body for the warps at a ragged row end or past the last row.
template <typename ST, int BC, int NZM, int W, bool EXACT, bool DEEP = false>
__device__ __forceinline__ void heat_column_dispatch(const HeatArgs& a, int bx, int by, int bz = 0) {
    const int x0 = (bx * 32 + threadIdx.x) * W;
    const int y = by * blockDim.y + threadIdx.y;
    const int z0 = DEEP ? bz * NZM : 0;
    // every vector of the warp lies inside the row (no ragged end, no lane past it)
    const bool full_x = __all_sync(0xffffffffu, x0 + W <= a.nx);
    // ... and none touches the row's first or last cell (Dirichlet-0 only)
    const bool inner_x = __all_sync(0xffffffffu, x0 > 0 && x0 + W < a.nx);
    if (full_x && y < a.ny) heat_column_body<ST, BC, NZM, W, EXACT, true, DEEP>(a, x0, y, z0, full_x, inner_x);
    else heat_column_body<ST, BC, NZM, W, EXACT, false, DEEP>(a, x0, y, z0, full_x, inner_x);
}

// The COLUMN tile of a 2D depth-1 step (the multi-instance kernel's COLUMN
// work item).
template <typename ST, int BC, int NZM, int W>
__device__ __forceinline__ void heat_column_tile(const HeatArgs& a, int bx, int by) {
    static_assert(NZM == 1, "multi-instance grids are 2D");
    heat_column_dispatch<ST, BC, 1, W, true>(a, bx, by);
}

// At most 256 threads per block and two blocks per SM: 128 registers a
// thread, which the 3D column (three arrays of eight planes x four cells)
// needs without spilling, and one wave of blocks at 512 x 512 x 8.  EXACT
// kernels serve nz == NZM (2D, and 3D stacks of 2, 4 or 8 planes); the
// general one (NZM = 8), every other nz <= 8 (separate kernels: one holding
// both paths spills).  DEEP kernels serve nz > 8: blockIdx.z picks a chunk
// of 8 planes, which the thread updates with the planes just below and
// above it as halos (EXACT when 8 divides nz).
template <typename ST, int BC, int NZM, int W, bool EXACT, bool DEEP>
__global__ void __launch_bounds__(256, 2) heat_column_kernel(const HeatArgs a) {
    pdl_wait_then_trigger();
    const uint3 b = block_index(a.rev);
    heat_column_dispatch<ST, BC, NZM, W, EXACT, DEEP>(a, b.x, b.y, b.z);
}

// ------------------------------------------- column, rows in shared memory --
//
// COLUMN with the y-neighbour rows staged in shared memory: each thread loads
// only its own row of every plane (the block's first and last thread rows
// also load the halo rows above and below the block), stores it to shared
// memory, and after one barrier reads rows y-1 and y+1 from there.  Fewer
// registers and L2 requests than COLUMN; z-neighbours from registers, x by
// shuffle.  Block (32, rows); shared memory (rows + 2) x NZM x 32 x V floats.
template <typename ST, int BC, int NZM>
__global__ void __launch_bounds__(256) heat_scol_kernel(const HeatArgs a) {
    constexpr int V = Vec<ST>::N;
    extern __shared__ float ssm[];
    pdl_wait_then_trigger();
    const int lane = threadIdx.x, ty = threadIdx.y, BY = blockDim.y;
    const uint3 blk = block_index(a.rev);
    const int x0 = (blk.x * 32 + lane) * V;
    const int y0 = blk.y * BY;
    const int y = y0 + ty;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool xin = x0 < nx;
    const bool act = xin && (y < ny);
    const bool fast_x = __all_sync(0xffffffffu, x0 > 0 && x0 + V < nx);
    const long long pitch = a.pitch, plane = a.plane;
    const ST* __restrict__ Tin = static_cast<const ST*>(a.Tin);
    const ST* base = Tin + (long long)min(y, ny - 1) * pitch + x0;
    const int slabf = 32 * V;  // floats of one (row, plane) slab
    float* mine = ssm + lane * V;

    float c[NZM][V], p[V], wl[NZM], er[NZM];
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
        wl[z] = 0.f;
        er[z] = 0.f;
#pragma unroll
        for (int i = 0; i < V; ++i) c[z][i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < V; ++i) p[i] = 0.f;
    if (act) {
#pragma unroll
        for (int z = 0; z < NZM; ++z) {
            if (z < nz) {
                const ST* q = base + z * plane;
                load_vec(q, c[z]);
                if (lane == 0 && x0 > 0) wl[z] = load_scalar(q - 1);
                if (lane == 31 && x0 + V < nx) er[z] = load_scalar(q + V);
            }
        }
        load_vec(static_cast<const ST*>(a.P) + (long long)y * a.p_pitch + x0, p);
    }
    // halo rows, each with its own condition (with one thread row per block
    // the same thread loads both): y0 - 1 into slab row 0 when it exists,
    // y0 + BY into slab row BY + 1 when it exists
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const bool want = side == 0 ? (ty == 0 && y0 > 0) : (ty == BY - 1 && y0 + BY < ny);
        if (!(xin && want)) continue;
        const int hy = side == 0 ? y0 - 1 : y0 + BY;
        const int hr = side == 0 ? 0 : BY + 1;
        const ST* hb = Tin + (long long)hy * pitch + x0;
#pragma unroll
        for (int z = 0; z < NZM; ++z) {
            if (z < nz) {
                float h[V];
                load_vec(hb + z * plane, h);
                sm_put<V>(mine + ((size_t)hr * NZM + z) * slabf, h);
            }
        }
    }
    if (act) {
#pragma unroll
        for (int z = 0; z < NZM; ++z)
            if (z < nz) sm_put<V>(mine + ((size_t)(ty + 1) * NZM + z) * slabf, c[z]);
    }
    __syncthreads();
#pragma unroll
    for (int z = 0; z < NZM; ++z) {
        if (z < nz) {  // warp-uniform
            float w0 = __shfl_up_sync(0xffffffffu, c[z][V - 1], 1);
            float eV = __shfl_down_sync(0xffffffffu, c[z][0], 1);
            if (lane == 0) w0 = wl[z];
            if (lane == 31) eV = er[z];
            if (!act) continue;
            float nv[V], sv[V];
            if (y > 0) sm_get<V>(mine + ((size_t)ty * NZM + z) * slabf, nv);
            else
#pragma unroll
                for (int i = 0; i < V; ++i) nv[i] = bnd<BC>(c[z][i]);
            if (y + 1 < ny) sm_get<V>(mine + ((size_t)(ty + 2) * NZM + z) * slabf, sv);
            else
#pragma unroll
                for (int i = 0; i < V; ++i) sv[i] = bnd<BC>(c[z][i]);
            float out[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const float t = c[z][i];
                float w = (i == 0) ? w0 : c[z][i - 1];
                float e = (i == V - 1) ? eV : c[z][i + 1];
                if (!fast_x) {
                    if (x0 + i == 0) w = bnd<BC>(t);
                    if (x0 + i + 1 >= nx) e = bnd<BC>(t);
                }
                float d = 0.f, u = 0.f;
                if (NZM > 1) {
                    d = (z > 0) ? c[z > 0 ? z - 1 : 0][i] : bnd<BC>(t);
                    u = (z + 1 < nz) ? c[z + 1 < NZM ? z + 1 : z][i] : bnd<BC>(t);
                }
                out[i] = heat_cell<(NZM > 1)>(t, nv[i], sv[i], w, e, d, u, (z == 0) ? p[i] : 0.0f, a.c);
            }
            store_vec(static_cast<ST*>(a.Tout) + (long long)z * plane + (long long)y * pitch + x0, out,
                      fast_x ? V : nx - x0);
        }
    }
}

// ------------------------------------------------------------ wavefront --
//
// Temporal blocking without shared-memory tiles: each warp owns 32 vectors
// of V cells along x (lanes 0 and 31 are halo lanes: loaded and computed but
// never stored, so the stored span of a warp is 30*V cells and neighbouring
// warps overlap by one vector on each side) and marches rows in y.  For
// every time level s = 0..T-1 a thread keeps a 3-row window of its vector in
// registers; at march step j (level-0 row r) level s computes row r - s from
// level s-1's window, so one pass over the rows advances T steps.  The halo
// lanes absorb the one cell of validity lost per level at each warp edge
// (requires T <= V).  In 3D the block holds all nz planes (one warp row per
// plane) and exchanges each level's newest row through a double-buffered
// shared-memory row, with one barrier per march step.  A block marches
// R + 2T level-0 rows to produce R output rows.  The kernel is bound by
// instruction issue: rows and tiles away from the grid's edges (a
// warp-uniform test) update with no boundary selects and packed f32x2
// arithmetic.
//
// Launch: 3D: block (32, nz), grid (x tiles, ceil(ny/R)).
//         2D: block (32, WB) with WB independent warps stacked in y,
//             grid (x tiles, ceil(ny/(R*WB))).
template <typename ST, int BC, bool IS3D, int T>
__global__ void __launch_bounds__(512) heat_wave_kernel(const HeatArgs a) {
    constexpr int V = Vec<ST>::N;
    static_assert(T >= 1 && T <= V, "halo lane must cover T cells");
    extern __shared__ float wsm[];  // 3D: [2][T][nz][32*V]
    pdl_wait_then_trigger();

    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int R = a.rows;
    const int stride = 30 * V;
    const uint3 blk = block_index(a.rev);
    const int xs = (int)blk.x * stride - V;      // global x of lane 0, element 0
    const int x0 = xs + lane * V;                 // this lane's first cell
    const int tz = IS3D ? (int)threadIdx.y : 0;
    const int nz = IS3D ? a.nz : 1;
    const int y0 = IS3D ? (int)blk.y * R : ((int)blk.y * (int)blockDim.y + (int)threadIdx.y) * R;
    const bool has_p = !IS3D || tz == 0;
    const bool ld_ok = (x0 >= 0) && (x0 < nx);   // vector lies (at least partly) in the grid
    const bool st_lane = (lane >= 1) && (lane <= 30) && (x0 < nx);
    const int rowlen = 32 * V;
    // the block's 32 vectors lie inside the row, away from both x edges
    // (every cell has both x-neighbours in the grid)
    const bool x_fast = (xs >= 1) && (xs + 32 * V < nx);

    const ST* __restrict__ Tin = static_cast<const ST*>(a.Tin);
    ST* __restrict__ Tout = static_cast<ST*>(a.Tout);
    const ST* __restrict__ P = static_cast<const ST*>(a.P);
    const long long zoff = IS3D ? (long long)tz * a.plane : 0;
    const ST* col = Tin + zoff + x0;
    const ST* pcol = P + x0;

    float win[T][3][V];
    float pr[T + 1][V];
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < V; ++i) win[s][k][i] = 0.f;
#pragma unroll
    for (int s = 0; s <= T; ++s)
#pragma unroll
        for (int i = 0; i < V; ++i) pr[s][i] = 0.f;

    // prefetch of level-0 row r (and its P row)
    float nrow[V], nprow[V];
    const int rbeg = y0 - T;
    const int nsteps = R + 2 * T;
#pragma unroll
    for (int i = 0; i < V; ++i) { nrow[i] = 0.f; nprow[i] = 0.f; }
    if (ld_ok && rbeg >= 0 && rbeg < ny) {
        load_vec(col + (long long)rbeg * a.pitch, nrow);
        if (has_p) load_vec(pcol + (long long)rbeg * a.p_pitch, nprow);
    }

    for (int j = 0; j < nsteps; ++j) {
        const int r = rbeg + j;
        // shift in level-0 row r, issue the load of row r+1
#pragma unroll
        for (int i = 0; i < V; ++i) {
            win[0][0][i] = win[0][1][i];
            win[0][1][i] = win[0][2][i];
            win[0][2][i] = nrow[i];
        }
#pragma unroll
        for (int s = T; s >= 1; --s)
#pragma unroll
            for (int i = 0; i < V; ++i) pr[s][i] = pr[s - 1][i];
#pragma unroll
        for (int i = 0; i < V; ++i) pr[0][i] = nprow[i];
#pragma unroll
        for (int i = 0; i < V; ++i) { nrow[i] = 0.f; nprow[i] = 0.f; }
        if (ld_ok && r + 1 >= 0 && r + 1 < ny && j + 1 < nsteps) {
            load_vec(col + (long long)(r + 1) * a.pitch, nrow);
            if (has_p) load_vec(pcol + (long long)(r + 1) * a.p_pitch, nprow);
        }

        float* wbuf = nullptr;
        const float* rbuf = nullptr;
        if (IS3D) {
            wbuf = wsm + (size_t)(j & 1) * T * nz * rowlen + lane * V;
            rbuf = wsm + (size_t)((j + 1) & 1) * T * nz * rowlen + lane * V;
            // After this barrier every thread has finished step j-1 (whose
            // reads used buffer j&1) and the rows written at step j-1 (into
            // buffer (j-1)&1) are visible.
            __syncthreads();
            sm_put<V>(wbuf + (size_t)tz * rowlen, win[0][2]);  // level 0, row r
        }

#pragma unroll
        for (int s = 1; s <= T; ++s) {
            const int q = r - s;  // row computed at this level
            const float(&c)[V] = win[s - 1][1];
            float w0 = __shfl_up_sync(0xffffffffu, c[V - 1], 1);
            float eV = __shfl_down_sync(0xffffffffu, c[0], 1);
            float dv[V], uv[V];
            if (IS3D) {
                const float* lv = rbuf + (size_t)(s - 1) * nz * rowlen;
                if (tz > 0) sm_get<V>(lv + (size_t)(tz - 1) * rowlen, dv);
                if (tz + 1 < nz) sm_get<V>(lv + (size_t)(tz + 1) * rowlen, uv);
            }
            float out[V];
            if (x_fast && q >= 1 && q + 1 < ny) {  // warp-uniform: no boundary within reach
                float xs[V], dd[V], uu[V], pp[V];
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    xs[i] = __fadd_rn((i == 0) ? w0 : c[i - 1], (i == V - 1) ? eV : c[i + 1]);
                    dd[i] = uu[i] = 0.f;
                    if (IS3D) {
                        dd[i] = (tz > 0) ? dv[i] : bnd<BC>(c[i]);
                        uu[i] = (tz + 1 < nz) ? uv[i] : bnd<BC>(c[i]);
                    }
                    pp[i] = has_p ? pr[s][i] : 0.0f;
                }
#pragma unroll
                for (int i = 0; i < V; i += 2)
                    heat_cell_x2<IS3D>(&c[i], &win[s - 1][0][i], &win[s - 1][2][i], &xs[i], &dd[i], &uu[i], &pp[i],
                                       a.c, &out[i]);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const int x = x0 + i;
                    const float t = c[i];
                    float w = (i == 0) ? w0 : c[i - 1];
                    float e = (i == V - 1) ? eV : c[i + 1];
                    if (x == 0) w = bnd<BC>(t);
                    if (x + 1 >= nx) e = bnd<BC>(t);
                    const float n = (q == 0) ? bnd<BC>(t) : win[s - 1][0][i];
                    const float so = (q + 1 >= ny) ? bnd<BC>(t) : win[s - 1][2][i];
                    float d = 0.f, u = 0.f;
                    if (IS3D) {
                        d = (tz > 0) ? dv[i] : bnd<BC>(t);
                        u = (tz + 1 < nz) ? uv[i] : bnd<BC>(t);
                    }
                    out[i] = heat_cell<IS3D>(t, n, so, w, e, d, u, has_p ? pr[s][i] : 0.0f, a.c);
                }
            }
            if (s < T) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    win[s][0][i] = win[s][1][i];
                    win[s][1][i] = win[s][2][i];
                    win[s][2][i] = out[i] = as_stored<ST>(out[i]);
                }
                if (IS3D) sm_put<V>(wbuf + ((size_t)s * nz + tz) * rowlen, out);
            } else if (st_lane && q >= y0 && q < y0 + R && q < ny) {
                store_vec(Tout + zoff + (long long)q * a.pitch + x0, out, nx - x0);
            }
        }
    }
}

// ------------------------------------------------- column, depth T (2D) ----
//
// Temporal blocking without a march, for 2D grids: each thread owns V cells
// along x and R consecutive output rows.  It issues all of its loads at once
// (rows y0-T .. y0+R+T-1 of T and the P rows y0-T+1 .. y0+R+T-2, at clamped
// coordinates) and advances T levels in registers: level k updates array
// rows k .. R+2T-1-k in place, each from level k-1's rows above and below.
// x-neighbours come from shuffles; a warp edge loses one cell of validity per
// level, so lanes 0 and 31 are halo lanes (T <= V) and a warp stores lanes
// 1..30 (tiles of 30 V cells, overlapping by a vector on each side, as the
// wavefront kernel's).  Rows outside the grid are computed but only feed rows
// whose neighbour there is replaced by the boundary value.  Blocks away from
// every grid edge (warp-uniform) update without boundary selects in packed
// f32x2 arithmetic.  Block (32, BY): BY warps stacked in y.
template <typename ST, int BC, int T, int R>
__device__ __forceinline__ void heat_column_t_tile(const HeatArgs& a, int bx, int by) {
    constexpr int V = Vec<ST>::N;
    constexpr int NR = R + 2 * T;
    static_assert(T >= 1 && T <= V, "halo lane must cover T cells");
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int xs = bx * 30 * V - V;  // global x of lane 0, element 0
    const int x0 = xs + lane * V;    // this lane's first cell
    const int y0 = (by * (int)blockDim.y + (int)threadIdx.y) * R;
    const int xc = min(max(x0, 0), (nx - 1) / V * V);  // a vector inside the row
    const long long pitch = a.pitch;
    const ST* __restrict__ Tin = static_cast<const ST*>(a.Tin);
    const ST* __restrict__ P = static_cast<const ST*>(a.P);

    float row[NR][V], pr[NR - 2][V];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int yk = min(max(y0 - T + k, 0), ny - 1);
        load_vec(Tin + (long long)yk * pitch + xc, row[k]);
    }
#pragma unroll
    for (int k = 1; k < NR - 1; ++k) {
        const int yk = min(max(y0 - T + k, 0), ny - 1);
        load_vec(P + (long long)yk * a.p_pitch + xc, pr[k - 1]);
    }
    // the block's 32 vectors lie away from both x edges, and no row it
    // updates is the grid's first or last
    const bool fast = (xs >= 1) && (xs + 32 * V < nx) && (y0 >= T) && (y0 + R + T <= ny);

#pragma unroll
    for (int k = 1; k <= T; ++k) {
        float prev[V];  // level k-1 value of the row above the one being updated
#pragma unroll
        for (int i = 0; i < V; ++i) prev[i] = row[k - 1][i];
#pragma unroll
        for (int j = k; j <= NR - 1 - k; ++j) {
            const int yg = y0 - T + j;
            const float(&c)[V] = row[j];
            const float w0 = __shfl_up_sync(0xffffffffu, c[V - 1], 1);
            const float eV = __shfl_down_sync(0xffffffffu, c[0], 1);
            float out[V];
            if (fast) {
                float xsum[V], zero[V];
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    xsum[i] = __fadd_rn((i == 0) ? w0 : c[i - 1], (i == V - 1) ? eV : c[i + 1]);
                    zero[i] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < V; i += 2)
                    heat_cell_x2<false>(&c[i], &prev[i], &row[j + 1][i], &xsum[i], &zero[i], &zero[i], &pr[j - 1][i],
                                        a.c, &out[i]);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const int x = x0 + i;
                    const float t = c[i];
                    float w = (i == 0) ? w0 : c[i - 1];
                    float e = (i == V - 1) ? eV : c[i + 1];
                    if (x == 0) w = bnd<BC>(t);
                    if (x + 1 >= nx) e = bnd<BC>(t);
                    const float n = (yg == 0) ? bnd<BC>(t) : prev[i];
                    const float so = (yg + 1 >= ny) ? bnd<BC>(t) : row[j + 1][i];
                    out[i] = heat_cell<false>(t, n, so, w, e, 0.f, 0.f, pr[j - 1][i], a.c);
                }
            }
#pragma unroll
            for (int i = 0; i < V; ++i) {
                prev[i] = row[j][i];
                row[j][i] = as_stored<ST>(out[i]);
            }
        }
    }
    if (lane >= 1 && lane <= 30 && x0 < nx) {
#pragma unroll
        for (int j = T; j < T + R; ++j) {
            const int yg = y0 - T + j;
            if (yg < ny) store_vec(static_cast<ST*>(a.Tout) + (long long)yg * pitch + x0, row[j], nx - x0);
        }
    }
}

template <typename ST, int BC, int T, int R>
__global__ void __launch_bounds__(256) heat_column_t_kernel(const HeatArgs a) {
    pdl_wait_then_trigger();
    const uint3 blk = block_index(a.rev);
    heat_column_t_tile<ST, BC, T, R>(a, (int)blk.x, (int)blk.y);
}


// --------------------------------------------- column, depth T (3D) -------
//
// Temporal blocking for thin stacks (nz <= 8) without shared memory: each
// lane owns one cell along x at R consecutive output rows and every plane of
// the column, so all z-neighbours are in its registers.  One round of loads
// (rows y0-T .. y0+R+T-1 of every plane, and the P rows of plane 0, all at
// clamped coordinates), then T levels in place: level k updates array rows
// k .. R+2T-1-k of every plane from level k-1 values (the row above comes
// from `prev`, saved before it was overwritten).  x-neighbours come from
// shuffles; a warp edge loses one lane of validity per level, so lanes
// 0..T-1 and 32-T..31 are halo lanes and a warp stores 32-2T cells (tiles
// overlap by 2T cells).  One cell a lane (rather than a vector) keeps the
// R+2T rows of eight planes within the registers the launch bounds leave a
// thread (R = 4: two blocks of 256 threads per SM; R = 2: three).  Warps
// whose rows and cells lie away from every x and y edge (warp-uniform)
// update without boundary selects, in packed f32x2 arithmetic over pairs of
// planes (EXACT kernels: the z-boundaries are compile-time).  Measured
// alternative: two cells a lane with the stack split between the half-warps
// (one shfl.xor per row for the plane across the halves) ran 16 % slower on
// 512 x 512 x 8: the cross-half shuffle sits on every row's dependency chain.
// Block (32, BY).
template <typename ST, int BC, int NZM, bool EXACT, int T, int R>
__device__ __forceinline__ void heat_column3_t_tile(const HeatArgs& a, int bx, int by) {
    constexpr int NR = R + 2 * T;
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int nz = EXACT ? NZM : a.nz;
    const int xs = bx * (32 - 2 * T) - T;  // global x of lane 0
    const int x = xs + lane;
    const int xc = min(max(x, 0), nx - 1);
    const int y0 = (by * (int)blockDim.y + (int)threadIdx.y) * R;
    const long long pitch = a.pitch, plane = a.plane;
    const ST* __restrict__ Tin = static_cast<const ST*>(a.Tin);
    const ST* __restrict__ P = static_cast<const ST*>(a.P);

    float row[NR][NZM], pr[NR - 2];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int yk = min(max(y0 - T + k, 0), ny - 1);
#pragma unroll
        for (int z = 0; z < NZM; ++z) {
            const int zc = EXACT ? z : min(z, nz - 1);
            row[k][z] = load_scalar(Tin + (long long)zc * plane + (long long)yk * pitch + xc);
        }
    }
#pragma unroll
    for (int k = 1; k < NR - 1; ++k) {
        const int yk = min(max(y0 - T + k, 0), ny - 1);
        pr[k - 1] = load_scalar(P + (long long)yk * a.p_pitch + xc);
    }
    // the warp's 32 cells lie away from both x edges, and no row it updates
    // is the grid's first or last
    const bool fast = EXACT && (NZM % 2 == 0) && (xs >= 1) && (xs + 32 < nx) && (y0 >= T) && (y0 + R + T <= ny);

#pragma unroll
    for (int k = 1; k <= T; ++k) {
        float prev[NZM];  // level k-1 values of the row above the one being updated
#pragma unroll
        for (int z = 0; z < NZM; ++z) prev[z] = row[k - 1][z];
#pragma unroll
        for (int j = k; j <= NR - 1 - k; ++j) {
            const int yg = y0 - T + j;
            float out[NZM];
            if (fast) {
                float xsum[NZM], zsum[NZM], pz[NZM];
#pragma unroll
                for (int z = 0; z < NZM; ++z) {
                    const float t = row[j][z];
                    xsum[z] = __fadd_rn(__shfl_up_sync(0xffffffffu, t, 1), __shfl_down_sync(0xffffffffu, t, 1));
                    const float dn = (z > 0) ? row[j][z > 0 ? z - 1 : 0] : bnd<BC>(t);
                    const float up = (z + 1 < NZM) ? row[j][z + 1 < NZM ? z + 1 : z] : bnd<BC>(t);
                    zsum[z] = __fadd_rn(dn, up);
                    pz[z] = (z == 0) ? pr[j - 1] : 0.0f;
                }
#pragma unroll
                for (int z = 0; z < NZM; z += 2)
                    heat_cell_x2z(&row[j][z], &prev[z], &row[j + 1][z], &xsum[z], &zsum[z], &pz[z], a.c, &out[z]);
            } else {
#pragma unroll
                for (int z = 0; z < NZM; ++z) {
                    // shuffles outside any divergent branch: every lane takes part
                    const float t = row[j][z];
                    float w = __shfl_up_sync(0xffffffffu, t, 1);
                    float e = __shfl_down_sync(0xffffffffu, t, 1);
                    if (!EXACT && z >= nz) {
                        out[z] = t;
                        continue;
                    }
                    if (x == 0) w = bnd<BC>(t);
                    if (x + 1 >= nx) e = bnd<BC>(t);
                    const float n = (yg == 0) ? bnd<BC>(t) : prev[z];
                    const float so = (yg + 1 >= ny) ? bnd<BC>(t) : row[j + 1][z];
                    const float d = (z == 0) ? bnd<BC>(t) : row[j][z > 0 ? z - 1 : 0];
                    float u = (z + 1 < NZM) ? row[j][z + 1 < NZM ? z + 1 : z] : bnd<BC>(t);
                    if (!EXACT && z + 1 >= nz) u = bnd<BC>(t);
                    out[z] = heat_cell<true>(t, n, so, w, e, d, u, (z == 0) ? pr[j - 1] : 0.0f, a.c);
                }
            }
#pragma unroll
            for (int z = 0; z < NZM; ++z) {
                prev[z] = row[j][z];
                row[j][z] = as_stored<ST>(out[z]);
            }
        }
    }
    if (lane >= T && lane < 32 - T && x < nx) {
        ST* out_p = static_cast<ST*>(a.Tout);
#pragma unroll
        for (int j = T; j < T + R; ++j) {
            const int yg = y0 - T + j;
            if (yg >= ny) break;
#pragma unroll
            for (int z = 0; z < NZM; ++z) {
                if (!EXACT && z >= nz) break;
                store_scalar(out_p + (long long)z * plane + (long long)yg * pitch + x, row[j][z]);
            }
        }
    }
}

// Rows per thread of the 3D depth-T COLUMN kernel: plan.rows 2 takes 2 (three
// blocks per SM), anything else the default, 4 at depth 2 and 2 at depth 4.
__host__ __device__ constexpr int column3_t_rows(int depth, int rows) {
    return (depth == 2 && rows != 2) ? 4 : 2;
}

template <typename ST, int BC, int NZM, bool EXACT, int T, int R>
__global__ void __launch_bounds__(256, R == 2 && T == 2 ? 3 : 2) heat_column3_t_kernel(const HeatArgs a) {
    pdl_wait_then_trigger();
    const uint3 blk = block_index(a.rev);
    heat_column3_t_tile<ST, BC, NZM, EXACT, T, R>(a, (int)blk.x, (int)blk.y);
}

// ------------------------------------------- z-march, depth 2 (deep 3D) ----
//
// Temporal blocking for deep stacks (nz > 8), where one step streams the
// whole field from DRAM: a block marches a chunk of tile_y planes in z and
// advances them two levels, reading T once and writing it once per two
// steps.  Each lane owns two cells along x (an 8-byte f32 or 4-byte bf16/f16
// access) at the R = 4 output rows of its warp; it keeps three planes of
// level 0 (rows y0-2 .. y0+5) and three of level 1 (rows y0-1 .. y0+4) in
// registers (the P rows, used on plane 0 only, are loaded there).  Level-0
// plane z completes level 1 of plane z-1 and then level 2 of plane z-2,
// which is stored.  The march is unrolled three times so that the window
// slots are compile-time.  Measured on 256^3 (GB300): 132 us per two-step
// launch against 20.8 us per depth-1 step of the chunked COLUMN kernel, so
// it loses to depth 1 there: 49 M instructions a launch (the boundary
// path runs in every warp touching an x or y edge, and 256 = 4 x 60 + 16
// leaves a mostly idle fifth tile), 38 % issue activity, and loading the
// next plane one step ahead (a fourth slot, 168 registers, 1.4 waves) did not
// change the time.  It is correct and tested, and kept as a plan.  x-neighbours by
// shuffle: a warp edge loses one cell per level, so lanes 0 and 31 are halo
// lanes (a warp stores 60 cells; tiles overlap by two on each side).  Rows
// and planes outside the grid are loaded at clamped coordinates and only
// feed values that the boundary rule replaces.  Warps away from the x and y
// edges update planes away from the z edges without selects, in packed
// f32x2 arithmetic on the lane's cell pair.  Block (32, BY), BY <= 4.
constexpr int kZmW = 2, kZmR = 4;

// One level on one plane: input rows 0 .. NI-1 of the plane below (B),
// itself (M) and above (A), at global rows yb .. yb+NI-1, give output rows
// 1 .. NI-2 (into out[0 .. NI-3]).  On plane 0 the P row of each output row
// is loaded where it is used (xc: the lane's clamped pair).
template <typename ST, int BC, int NI>
__device__ __forceinline__ void zm_level(const HeatArgs& a, int p, int yb, int x0, int xc, bool fast_xy,
                                         const float (&B)[NI][kZmW], const float (&M)[NI][kZmW],
                                         const float (&A)[NI][kZmW], float (&out)[NI - 2][kZmW]) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool fast = fast_xy && p > 0 && p + 1 < nz;  // warp-uniform
#pragma unroll
    for (int i = 1; i <= NI - 2; ++i) {
        const float(&t)[kZmW] = M[i];
        const float w0 = __shfl_up_sync(0xffffffffu, t[kZmW - 1], 1);
        const float eW = __shfl_down_sync(0xffffffffu, t[0], 1);
        if (fast) {
            float xsum[kZmW], zero[kZmW] = {0.0f, 0.0f};
            xsum[0] = __fadd_rn(w0, t[1]);
            xsum[1] = __fadd_rn(t[0], eW);
            heat_cell_x2<true>(t, M[i - 1], M[i + 1], xsum, B[i], A[i], zero, a.c, out[i - 1]);
        } else {
            const int yg = yb + i;
            float pz[kZmW] = {0.0f, 0.0f};
            if (p == 0)
                load_vecw<ST, kZmW>(static_cast<const ST*>(a.P) + (long long)min(max(yg, 0), ny - 1) * a.p_pitch + xc,
                                    pz);
#pragma unroll
            for (int c = 0; c < kZmW; ++c) {
                const int x = x0 + c;
                const float tc = t[c];
                float w = (c == 0) ? w0 : t[c - 1];
                float e = (c == kZmW - 1) ? eW : t[c + 1];
                if (x == 0) w = bnd<BC>(tc);
                if (x + 1 >= nx) e = bnd<BC>(tc);
                const float n = (yg == 0) ? bnd<BC>(tc) : M[i - 1][c];
                const float so = (yg + 1 >= ny) ? bnd<BC>(tc) : M[i + 1][c];
                const float d = (p == 0) ? bnd<BC>(tc) : B[i][c];
                const float u = (p + 1 >= nz) ? bnd<BC>(tc) : A[i][c];
                out[i - 1][c] = heat_cell<true>(tc, n, so, w, e, d, u, pz[c], a.c);
            }
        }
#pragma unroll
        for (int c = 0; c < kZmW; ++c) out[i - 1][c] = as_stored<ST>(out[i - 1][c]);
    }
}

template <typename ST>
__device__ __forceinline__ void zm_load(const HeatArgs& a, int z, int y0, int xc, float (&L)[kZmR + 4][kZmW]) {
    const ST* __restrict__ base = static_cast<const ST*>(a.Tin) + (long long)z * a.plane + xc;
#pragma unroll
    for (int k = 0; k < kZmR + 4; ++k) {
        const int yk = min(max(y0 - 2 + k, 0), a.ny - 1);
        load_vecw<ST, kZmW>(base + (long long)yk * a.pitch, L[k]);
    }
}

// Step r of the march (PH = r mod 3): level-0 plane z = zs + r arrives,
// level 1 of plane z-1 and level 2 of plane z-2 follow.
template <typename ST, int BC, int PH>
__device__ __forceinline__ void zm_step(const HeatArgs& a, int r, int zs, int z0, int z1, int y0, int x0, int xc,
                                        bool fast_xy, bool store_lane, float (&L0)[3][kZmR + 4][kZmW],
                                        float (&L1)[3][kZmR + 2][kZmW]) {
    constexpr int S0 = PH, S1 = (PH + 1) % 3, S2 = (PH + 2) % 3;  // slots of planes z, z-2, z-1
    const int nz = a.nz;
    const int z = zs + r;
    if (z >= 0 && z < nz) zm_load<ST>(a, z, y0, xc, L0[S0]);
    const int p1 = z - 1;
    if (p1 >= max(z0 - 1, 0) && p1 <= min(z1, nz - 1))
        zm_level<ST, BC, kZmR + 4>(a, p1, y0 - 2, x0, xc, fast_xy, L0[S1], L0[S2], L0[S0], L1[S2]);
    const int p2 = z - 2;
    if (p2 >= z0 && p2 < z1) {
        float out[kZmR][kZmW];
        zm_level<ST, BC, kZmR + 2>(a, p2, y0 - 1, x0, xc, fast_xy, L1[S0], L1[S1], L1[S2], out);
        if (store_lane) {
            ST* o = static_cast<ST*>(a.Tout) + (long long)p2 * a.plane + x0;
            const int nv = min(kZmW, a.nx - x0);
#pragma unroll
            for (int i = 0; i < kZmR; ++i) {
                const int yg = y0 + i;
                if (yg < a.ny) store_vecw<ST, kZmW>(o + (long long)yg * a.pitch, out[i], nv);
            }
        }
    }
}

template <typename ST, int BC>
__global__ void __launch_bounds__(128, 4) heat_zmarch2_kernel(const HeatArgs a) {
    pdl_wait_then_trigger();
    const uint3 blk = block_index(a.rev);
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xs = (int)blk.x * (30 * kZmW) - kZmW;  // global x of lane 0's first cell
    const int x0 = xs + lane * kZmW;
    const int xc = min(max(x0, 0), (nx - 1) / kZmW * kZmW);
    const int y0 = ((int)blk.y * (int)blockDim.y + (int)threadIdx.y) * kZmR;
    const int z0 = (int)blk.z * a.tile_y;
    const int z1 = min(z0 + a.tile_y, nz);
    // every cell of the warp away from both x edges, no level-1 row on a y edge
    const bool fast_xy = (xs >= 1) && (xs + 32 * kZmW < nx) && (y0 >= 2) && (y0 + kZmR + 2 <= ny);
    const bool store_lane = lane >= 1 && lane <= 30 && x0 < nx;
    float L0[3][kZmR + 4][kZmW], L1[3][kZmR + 2][kZmW];
    const int zs = z0 - 2;
    const int rend = z1 + 2 - zs;  // level-0 planes zs .. z1+1
    for (int r = 0; r < rend; r += 3) {
        zm_step<ST, BC, 0>(a, r, zs, z0, z1, y0, x0, xc, fast_xy, store_lane, L0, L1);
        if (r + 1 < rend) zm_step<ST, BC, 1>(a, r + 1, zs, z0, z1, y0, x0, xc, fast_xy, store_lane, L0, L1);
        if (r + 2 < rend) zm_step<ST, BC, 2>(a, r + 2, zs, z0, z1, y0, x0, xc, fast_xy, store_lane, L0, L1);
    }
}

// ------------------------------------------------- STREAM (TMA z-march) ----
//
// Temporal depth 2 for 3D stacks: a march along z through shared memory, fed
// by the Tensor Memory Accelerator.  A block owns an x-y tile of 128 stored
// cells along x and 2W - 2 stored rows (W compute warps, each lane four
// cells along x at two rows) and a chunk of `tile_y` planes.  The tile's
// level-0 planes, with a halo of two rows and one 16-byte unit of columns on
// each side, stream through a ring of kStreamStages shared-memory stages
// (one cp.async.bulk.tensor box per plane, its completion counted on the
// stage's mbarrier).  For each arriving plane z the block computes level 1
// of plane z-1 into one of two shared level-1 planes and level 2 of plane
// z-2, which it stores.  A thread keeps its own cells' last three level-1
// planes in registers; x/y neighbours come from shared memory (x: within a
// lane's four cells, by shuffle between lanes, and from the halo columns at
// the warp's edges).  One extra warp computes the level-1 cells of the two
// halo columns (x0-1 and x0+128) and issues the copies.  One barrier per
// plane.  Each wait on a stage is bounded by kStreamWaitNs of the global
// timer: on a time-out the block stops, counts it in g_stream_timeouts and
// returns after its copies in flight have landed (waits bounded the same
// way); its stores are then incomplete.
constexpr int kStreamTileX = 128;  // stored cells along x per block (32 lanes x 4)
constexpr int kStreamRows = 2;     // level-1 rows per compute thread
constexpr int kStreamStages = 6;   // level-0 planes in the shared ring
constexpr unsigned long long kStreamWaitNs = 1000000000ull;

__device__ unsigned int g_stream_timeouts;

template <typename ST>
__host__ __device__ constexpr int stream_pad() { return 16 / (int)sizeof(ST); }  // halo columns on each side of a stage row
template <typename ST>
__host__ __device__ constexpr int stream_cols() { return kStreamTileX + 2 * stream_pad<ST>(); }
__host__ __device__ constexpr size_t stream_align128(size_t b) { return (b + 127) / 128 * 128; }
template <typename ST>
__host__ __device__ constexpr size_t stream_stage_bytes(int W) { return stream_align128((size_t)(2 * W + 2) * stream_cols<ST>() * sizeof(ST)); }
template <typename ST>
__host__ __device__ constexpr size_t stream_smem(int W) {
    return kStreamStages * stream_stage_bytes<ST>(W) + (size_t)2 * (2 * W) * stream_cols<ST>() * sizeof(float) +
           kStreamStages * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of `parity` to complete, for at most kStreamWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < kStreamWaitNs)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// One box of the tensor map at (x, y, z) into shared memory; completion is
// counted on `bar` (which the issuing thread armed with the box's bytes).
__device__ __forceinline__ void tma_load_plane(void* dst, const CUtensorMap* map, int x, int y, int z,
                                               unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Four consecutive cells of a shared stage row (16 bytes in f32, 8 in 16-bit types).
template <typename ST>
__device__ __forceinline__ void stage_get4(const ST* p, float (&v)[4]) {
    if constexpr (sizeof(ST) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const uint2 raw = *reinterpret_cast<const uint2*>(p);
        const ST* e = reinterpret_cast<const ST*>(&raw);
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = to_f32(e[i]);
    }
}
__device__ __forceinline__ void l1_get4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void l1_put4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Four cells of one row: own values t, rows n / so, planes d / u, the
// x-neighbours wv (left of cell 0) and ev (right of cell 3), both already
// under the boundary rule at the tile's outer edges.  `edge` (warp-uniform):
// the row is the grid's first or last row or lies outside it, the plane is
// the first or last, or the tile ends inside the row; then the boundary rule
// replaces each missing neighbour and plane 0 adds P.  The arithmetic is
// heat_cell's, in packed pairs either way.
template <typename ST, int BC>
__device__ __forceinline__ void stream_row(bool edge, const float (&t)[4], const float (&n)[4], const float (&so)[4],
                                           const float (&d)[4], const float (&u)[4], float wv, float ev, int x, int y,
                                           int p, const HeatArgs& a, float (&out)[4]) {
    float xs[4];
    if (!edge) {
        float zero[2] = {0.0f, 0.0f};
        xs[0] = __fadd_rn(wv, t[1]);
        xs[1] = __fadd_rn(t[0], t[2]);
        xs[2] = __fadd_rn(t[1], t[3]);
        xs[3] = __fadd_rn(t[2], ev);
        heat_cell_x2<true>(t, n, so, xs, d, u, zero, a.c, out);
        heat_cell_x2<true>(t + 2, n + 2, so + 2, xs + 2, d + 2, u + 2, zero, a.c, out + 2);
    } else {
        const int nx = a.nx, ny = a.ny, nz = a.nz;
        const bool top = (y == 0), bot = (y + 1 >= ny), lo = (p == 0), hi = (p + 1 >= nz);
        float nn[4], ss[4], dd[4], uu[4], pw[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float w = (c == 0) ? wv : t[c - 1];
            const float e = (x + c + 1 >= nx) ? bnd<BC>(t[c]) : (c == 3 ? ev : t[c + 1]);
            xs[c] = __fadd_rn(w, e);
            nn[c] = top ? bnd<BC>(t[c]) : n[c];
            ss[c] = bot ? bnd<BC>(t[c]) : so[c];
            dd[c] = lo ? bnd<BC>(t[c]) : d[c];
            uu[c] = hi ? bnd<BC>(t[c]) : u[c];
        }
        if (lo) {
            const ST* prow = static_cast<const ST*>(a.P) + (long long)min(max(y, 0), ny - 1) * a.p_pitch;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (x + c < nx) pw[c] = load_scalar_rw<ST>(prow + x + c);
        }
        heat_cell_x2<true>(t, nn, ss, xs, dd, uu, pw, a.c, out);
        heat_cell_x2<true>(t + 2, nn + 2, ss + 2, xs + 2, dd + 2, uu + 2, pw + 2, a.c, out + 2);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = as_stored<ST>(out[c]);
}

struct StreamArgs {
    CUtensorMap map;  // Tin as (nx, ny, nz) elements, box (stream_cols, 2W + 2, 1); sets the alignment
    HeatArgs a;
};

// What one step of a block's march needs besides the thread's own state:
// shared-memory offsets of the three level-0 stages (planes p1-1, p1, p1+1)
// and the two level-1 planes (written: p1, read: p2 = p1-1), the planes, and
// which of the two levels the step computes.
struct StreamStep {
    unsigned lo, mid, hi, l1w, l1r;  // byte offsets into the block's shared memory
    int p1, p2;
    bool do1, do2;
};

// What a thread of the march keeps for every step: `tb`, its element
// offset in a stage or level-1 plane (row 2w, column PX + 4 lane); `eb`, the
// same at column PX; `gout`, its first cell of level-2 output row
// y0 - 1 + 2w (plane 0); `x`, its first cell's column; `fast_x`: the tile
// ends at or before the row's end; lane0 / lane31: the lane takes its outer
// x-neighbour from the halo column, wfix / efix: that neighbour is outside
// the grid; row_edge[k]: row k needs the boundary rule in y; store_row[k]:
// row k is a stored level-2 row.
template <typename ST>
struct StreamThread {
    int tb, eb, x;
    ST* gout;
    bool fast_x, lane0, lane31, wfix, efix;
    bool row_edge[kStreamRows], store_row[kStreamRows];
};

// The x-neighbours left of cell 0 and right of cell 3 of a lane's four
// cells: the neighbour lanes' cells, at the warp's ends the halo column's
// (wl, er), and the boundary rule at the grid's ends.
template <int BC, typename ST>
__device__ __forceinline__ void stream_xnb(const StreamThread<ST>& th, const float (&t)[4], float wl, float er,
                                           float& wv, float& ev) {
    wv = __shfl_up_sync(0xffffffffu, t[3], 1);
    ev = __shfl_down_sync(0xffffffffu, t[0], 1);
    wv = th.lane0 ? wl : wv;
    ev = th.lane31 ? er : ev;
    wv = th.wfix ? bnd<BC>(t[0]) : wv;
    ev = th.efix ? bnd<BC>(t[3]) : ev;
}

// One step of the march (PH = step mod 3 names the register slots of the
// last three level-1 planes).
template <typename ST, int BC, int W, int PH>
__device__ __forceinline__ void stream_step(const StreamArgs& sa, unsigned char* smem, const StreamStep& st, int x0,
                                            int y0, const StreamThread<ST>& th, float (&ring)[3][kStreamRows][4]) {
    constexpr int PX = stream_pad<ST>(), BWC = stream_cols<ST>(), L1R = 2 * W;
    constexpr int S_NEW = PH, S_MID = (PH + 2) % 3, S_OLD = (PH + 1) % 3;  // slots of p1, p1-1, p1-2
    const HeatArgs& a = sa.a;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int nx = a.nx, nz = a.nz;
    const int tb = th.tb, eb = th.eb, x = th.x;
    const bool fast_x = th.fast_x;
    if (st.do1) {
        const ST* lo = reinterpret_cast<const ST*>(smem + st.lo);
        const ST* mid = reinterpret_cast<const ST*>(smem + st.mid);
        const ST* hi = reinterpret_cast<const ST*>(smem + st.hi);
        float* l1w = reinterpret_cast<float*>(smem + st.l1w);
        const int p1 = st.p1;
        if (w < W) {
            const bool zedge = !fast_x || p1 <= 0 || p1 + 1 >= nz;
            float rowv[kStreamRows + 2][4];
#pragma unroll
            for (int k = 0; k < kStreamRows + 2; ++k) stage_get4<ST>(mid + tb + k * BWC, rowv[k]);
#pragma unroll
            for (int k = 0; k < kStreamRows; ++k) {
                float d[4], u[4];
                stage_get4<ST>(lo + tb + (k + 1) * BWC, d);
                stage_get4<ST>(hi + tb + (k + 1) * BWC, u);
                const float(&t)[4] = rowv[k + 1];
                const float wl = to_f32(mid[eb + (k + 1) * BWC - 1]);             // x0-1 (broadcast)
                const float er = to_f32(mid[eb + (k + 1) * BWC + kStreamTileX]);  // x0+128
                float wv, ev;
                stream_xnb<BC>(th, t, wl, er, wv, ev);
                float out[4];
                stream_row<ST, BC>(zedge || th.row_edge[k], t, rowv[k], rowv[k + 2], d, u, wv, ev, x,
                                   y0 - 1 + w * kStreamRows + k, p1, a, out);
                l1_put4(l1w + tb + k * BWC, out);
#pragma unroll
                for (int c = 0; c < 4; ++c) ring[S_NEW][k][c] = out[c];
            }
        } else {
            // the halo columns x0-1 (j < L1R) and x0+128 at level-1 row i
            const int ny = a.ny;
#pragma unroll
            for (int j = lane; j < 2 * L1R; j += 32) {
                const int side = j >= L1R, i = side ? j - L1R : j, y = y0 - 1 + i;
                const int xh = side ? x0 + kStreamTileX : x0 - 1;
                if (xh < 0 || xh >= nx) continue;
                const int cc = side ? PX + kStreamTileX : PX - 1;
                const int o = (i + 1) * BWC + cc;
                const float tc = to_f32(mid[o]);
                const float wl = (xh == 0) ? bnd<BC>(tc) : to_f32(mid[o - 1]);
                const float er = (xh + 1 >= nx) ? bnd<BC>(tc) : to_f32(mid[o + 1]);
                const float nn = (y == 0) ? bnd<BC>(tc) : to_f32(mid[o - BWC]);
                const float ss = (y + 1 >= ny) ? bnd<BC>(tc) : to_f32(mid[o + BWC]);
                const float dd = (p1 == 0) ? bnd<BC>(tc) : to_f32(lo[o]);
                const float uu = (p1 + 1 >= nz) ? bnd<BC>(tc) : to_f32(hi[o]);
                float pw = 0.0f;
                if (p1 == 0)
                    pw = load_scalar_rw<ST>(static_cast<const ST*>(a.P) + (long long)min(max(y, 0), ny - 1) * a.p_pitch + xh);
                l1w[i * BWC + cc] = as_stored<ST>(heat_cell<true>(tc, nn, ss, wl, er, dd, uu, pw, a.c));
            }
        }
    }
    if (st.do2 && w < W) {
        const float* l1r = reinterpret_cast<const float*>(smem + st.l1r);  // level 1 of plane p2 (previous step)
        const int p2 = st.p2;
        const bool zedge = !fast_x || p2 <= 0 || p2 + 1 >= nz;
        ST* orow = th.gout + (long long)p2 * a.plane;
#pragma unroll
        for (int k = 0; k < kStreamRows; ++k) {
            if (!th.store_row[k]) continue;  // a halo row of level 1, or outside the grid (warp-uniform)
            const int y = y0 - 1 + w * kStreamRows + k;
            // rows i-1 / i+1: the thread's own other row from registers, the other from shared memory
            float nb[4], sb[4];
            if (k == 0) {
                l1_get4(l1r + tb - BWC, nb);
#pragma unroll
                for (int c = 0; c < 4; ++c) sb[c] = ring[S_MID][1][c];
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) nb[c] = ring[S_MID][0][c];
                l1_get4(l1r + tb + 2 * BWC, sb);
            }
            const float(&t)[4] = ring[S_MID][k];
            const float wl = l1r[eb + k * BWC - 1];
            const float er = l1r[eb + k * BWC + kStreamTileX];
            float wv, ev;
            stream_xnb<BC>(th, t, wl, er, wv, ev);
            float out[4];
            stream_row<ST, BC>(zedge || th.row_edge[k], t, nb, sb, ring[S_OLD][k], ring[S_NEW][k], wv, ev, x, y, p2,
                               a, out);
            if (fast_x)
                store_vecw<ST, 4>(orow + (long long)k * a.pitch, out, 4);
            else if (x < nx)
                store_vecw<ST, 4>(orow + (long long)k * a.pitch, out, nx - x);
        }
    }
}

template <typename ST, int BC, int W>
__global__ void __launch_bounds__(32 * (W + 1), W <= 8 ? 2 : 1) heat_stream2_kernel(const __grid_constant__ StreamArgs sa) {
    constexpr int PX = stream_pad<ST>(), BWC = stream_cols<ST>(), L1R = 2 * W;
    constexpr unsigned SB = (unsigned)stream_stage_bytes<ST>(W);
    constexpr unsigned L1B = (unsigned)(L1R * BWC * sizeof(float));  // one level-1 plane
    constexpr unsigned BOX_BYTES = (unsigned)((L1R + 2) * BWC * sizeof(ST));
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + kStreamStages * SB + 2 * L1B);
    const HeatArgs& a = sa.a;
    const uint3 blk = block_index(a.rev);
    const int x0 = (int)blk.x * kStreamTileX;
    const int y0 = (int)blk.y * (L1R - 2);
    const int z0 = (int)blk.z * a.tile_y;
    const int z1 = min(z0 + a.tile_y, a.nz);
    const int n0 = z1 - z0 + 4;  // level-0 planes z0-2 .. z1+1
    const int lane = threadIdx.x, w = threadIdx.y;
    const bool producer = w == W && lane == 0;
    StreamThread<ST> th;
    th.tb = w * kStreamRows * BWC + PX + 4 * lane;
    th.eb = w * kStreamRows * BWC + PX;
    th.x = x0 + 4 * lane;
    th.fast_x = x0 + kStreamTileX <= a.nx;
    th.lane0 = lane == 0;
    th.lane31 = lane == 31;
    th.wfix = lane == 0 && x0 == 0;
    th.efix = lane == 31 && x0 + kStreamTileX >= a.nx;
#pragma unroll
    for (int k = 0; k < kStreamRows; ++k) {
        const int i = w * kStreamRows + k, y = y0 - 1 + i;
        th.row_edge[k] = y <= 0 || y + 1 >= a.ny;
        th.store_row[k] = i >= 1 && i <= L1R - 2 && y < a.ny;
    }
    th.gout = static_cast<ST*>(a.Tout) + (long long)(y0 - 1 + w * kStreamRows) * a.pitch + x0 + 4 * lane;
    // level-1 planes start at zero (the halo columns outside the grid are
    // read, never used)
    {
        float* l1 = reinterpret_cast<float*>(smem + kStreamStages * SB);
        const int tid = w * 32 + lane;
        for (int e = tid; e < 2 * L1R * BWC; e += 32 * (W + 1)) l1[e] = 0.0f;
    }
    if (producer) {
        for (int s = 0; s < kStreamStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    pdl_wait_then_trigger();  // the previous step's stores are visible from here on
    if (producer) {
        for (int q = 0; q < kStreamStages && q < n0; ++q) {
            mbar_expect_tx(&bar[q], BOX_BYTES);
            tma_load_plane(smem + q * SB, &sa.map, x0 - PX, y0 - 2, z0 - 2 + q, &bar[q]);
        }
    }
    float ring[3][kStreamRows][4];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int k = 0; k < kStreamRows; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[s][k][c] = 0.0f;
    // steps whose level-1 plane p1 = z0-3+r is computed
    const int r1lo = max(2, max(z0 - 1, 0) - z0 + 3), r1hi = min(z1, a.nz - 1) - z0 + 3;
    int issued = min(kStreamStages, n0);
    bool failed = false;
    int si = 0;            // stage of plane r
    unsigned parity = 0;   // phase parity of that stage's fill
    StreamStep st;
    st.mid = (kStreamStages - 1) * SB;
    st.hi = 0;
    for (int r = 0; r < n0 && !failed; r += 3) {
#pragma unroll
        for (int ph = 0; ph < 3; ++ph) {
            const int rr = r + ph;
            if (rr >= n0 || failed) break;
            const bool ok = mbar_wait_bounded(&bar[si], parity);
            st.lo = st.mid;
            st.mid = st.hi;
            st.hi = si * SB;
            st.l1w = kStreamStages * SB + (rr & 1) * L1B;
            st.l1r = kStreamStages * SB + ((rr & 1) ^ 1) * L1B;
            st.p1 = z0 - 3 + rr;
            st.p2 = st.p1 - 1;
            st.do1 = rr >= r1lo && rr <= r1hi;
            st.do2 = rr >= 4;
            if (ph == 0) stream_step<ST, BC, W, 0>(sa, smem, st, x0, y0, th, ring);
            if (ph == 1) stream_step<ST, BC, W, 1>(sa, smem, st, x0, y0, th, ring);
            if (ph == 2) stream_step<ST, BC, W, 2>(sa, smem, st, x0, y0, th, ring);
            failed = __syncthreads_or(!ok) != 0;
            if (++si == kStreamStages) {
                si = 0;
                parity ^= 1u;
            }
            // the stage of plane rr-2 is free: refill it with plane rr-2+kStreamStages
            if (producer && !failed && rr >= 2 && issued < n0) {
                const int q = issued++;
                const unsigned sq = (unsigned)(q % kStreamStages);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar[sq], BOX_BYTES);
                tma_load_plane(smem + sq * SB, &sa.map, x0 - PX, y0 - 2, z0 - 2 + q, &bar[sq]);
            }
        }
    }
    if (failed && producer) {
        // let every copy in flight land before the block's shared memory is released
        for (int q = max(issued - kStreamStages, 0); q < issued; ++q)
            mbar_wait_bounded(&bar[q % kStreamStages], (unsigned)((q / kStreamStages) & 1));
        atomicAdd(&g_stream_timeouts, 1u);
    }
}

// ------------------------------------------------------------- factory ----

namespace {
template <int KIND>
const void* multi_func(gs_dtype dt, gs_bc bc) {
    const bool cl = (bc == GS_BC_CLAMP);
    switch (dt) {
        case GS_F32: return cl ? (const void*)heat_multi_kernel<float, GS_BC_CLAMP, KIND>
                               : (const void*)heat_multi_kernel<float, GS_BC_DIRICHLET0, KIND>;
        case GS_BF16: return cl ? (const void*)heat_multi_kernel<__nv_bfloat16, GS_BC_CLAMP, KIND>
                                : (const void*)heat_multi_kernel<__nv_bfloat16, GS_BC_DIRICHLET0, KIND>;
        case GS_F16: return cl ? (const void*)heat_multi_kernel<__half, GS_BC_CLAMP, KIND>
                               : (const void*)heat_multi_kernel<__half, GS_BC_DIRICHLET0, KIND>;
    }
    return nullptr;
}
}  // namespace

const void* heat_multi_func(gs_dtype dt, gs_bc bc, int variant, int depth) {
    if (variant != GS_KERNEL_COLUMN) return depth == 1 ? multi_func<0>(dt, bc) : nullptr;
    switch (depth) {
        case 1: return multi_func<1>(dt, bc);
        case 2: return multi_func<2>(dt, bc);
        case 4: return multi_func<4>(dt, bc);
    }
    return nullptr;
}

int heat_multi_span(gs_dtype dt, int variant, int depth, int block_x) {
    const int V = (dt == GS_F32) ? 4 : 8;
    if (variant != GS_KERNEL_COLUMN) return block_x * V;
    return depth > 1 ? 30 * V : 32 * V;
}

int heat_multi_item_rows(gs_dtype dt, int variant, int depth, int rows) {
    if (variant == GS_KERNEL_COLUMN && depth > 1)
        return rows * ((dt == GS_F32) ? column_t_rows<float>() : column_t_rows<__half>());
    return rows;
}

size_t heat_scol_smem(int nzm, int rows, int vec) { return (size_t)(rows + 2) * nzm * 32 * vec * sizeof(float); }

size_t heat_wave_smem(int nz3d, int depth, int vec) {
    return nz3d > 0 ? (size_t)2 * depth * nz3d * 32 * vec * sizeof(float) : 0;
}

size_t heat_temporal_smem(int nz, int tile_x, int tile_y, int depth) {
    const size_t area = (size_t)(tile_x + 2 * depth) * (tile_y + 2 * depth);
    return (2 * area * (size_t)nz + area) * sizeof(float);
}

namespace {

template <typename ST, int BC, bool IS3D>
const void* pick_temporal(int depth) {
    switch (depth) {
        case 2: return (const void*)heat_temporal_kernel<ST, BC, IS3D, 2>;
        case 4: return (const void*)heat_temporal_kernel<ST, BC, IS3D, 4>;
        default: return nullptr;
    }
}

template <typename ST, int BC, bool IS3D>
const void* pick_wave(int depth) {
    switch (depth) {
        case 1: return (const void*)heat_wave_kernel<ST, BC, IS3D, 1>;
        case 2: return (const void*)heat_wave_kernel<ST, BC, IS3D, 2>;
        case 4: return (const void*)heat_wave_kernel<ST, BC, IS3D, 4>;
        default: return nullptr;
    }
}

template <typename ST, int BC>
const void* pick(bool is3d, int depth, int variant, int nz, int rows) {
    if (variant == GS_KERNEL_COLUMN && depth == 1) {
        constexpr int W3 = column_width<ST>(true);
        if (!is3d) return (const void*)heat_column_kernel<ST, BC, 1, column_width<ST>(false), true, false>;
        if (nz > kColumnMaxNz)
            return nz % kColumnMaxNz == 0 ? (const void*)heat_column_kernel<ST, BC, kColumnMaxNz, W3, true, true>
                                          : (const void*)heat_column_kernel<ST, BC, kColumnMaxNz, W3, false, true>;
        switch (nz) {
            case 2: return (const void*)heat_column_kernel<ST, BC, 2, W3, true, false>;
            case 4: return (const void*)heat_column_kernel<ST, BC, 4, W3, true, false>;
            case kColumnMaxNz: return (const void*)heat_column_kernel<ST, BC, kColumnMaxNz, W3, true, false>;
            default: return (const void*)heat_column_kernel<ST, BC, kColumnMaxNz, W3, false, false>;
        }
    }
    if (variant == GS_KERNEL_COLUMN_SMEM && depth == 1)
        return is3d ? (const void*)heat_scol_kernel<ST, BC, kColumnMaxNz>
                    : (const void*)heat_scol_kernel<ST, BC, 1>;
    if (variant == GS_KERNEL_COLUMN && depth > 1 && !is3d) {
        if (depth == 2) return (const void*)heat_column_t_kernel<ST, BC, 2, column_t_rows<ST>()>;
        if (depth == 4) return (const void*)heat_column_t_kernel<ST, BC, 4, column_t_rows<ST>()>;
        return nullptr;
    }
    if (variant == GS_KERNEL_COLUMN && depth > 1 && is3d) {
        if (nz > kColumnMaxNz) return depth == 2 ? (const void*)heat_zmarch2_kernel<ST, BC> : nullptr;
        const bool exact8 = (nz == kColumnMaxNz);
        if (depth == 2 && rows == 2)
            return exact8 ? (const void*)heat_column3_t_kernel<ST, BC, kColumnMaxNz, true, 2, 2>
                          : (nz == 4 ? (const void*)heat_column3_t_kernel<ST, BC, 4, true, 2, 2>
                                     : (const void*)heat_column3_t_kernel<ST, BC, kColumnMaxNz, false, 2, 2>);
        if (depth == 2)
            return exact8 ? (const void*)heat_column3_t_kernel<ST, BC, kColumnMaxNz, true, 2, 4>
                          : (nz == 4 ? (const void*)heat_column3_t_kernel<ST, BC, 4, true, 2, 4>
                                     : (const void*)heat_column3_t_kernel<ST, BC, kColumnMaxNz, false, 2, 4>);
        if (depth == 4)
            return exact8 ? (const void*)heat_column3_t_kernel<ST, BC, kColumnMaxNz, true, 4, 2>
                          : (nz == 4 ? (const void*)heat_column3_t_kernel<ST, BC, 4, true, 4, 2>
                                     : (const void*)heat_column3_t_kernel<ST, BC, kColumnMaxNz, false, 4, 2>);
        return nullptr;
    }
    if (variant == GS_KERNEL_WAVE)
        return is3d ? pick_wave<ST, BC, true>(depth) : pick_wave<ST, BC, false>(depth);
    if (variant == GS_KERNEL_MARCH && depth == 1)
        return is3d ? (const void*)heat_step_kernel<ST, BC, true> : (const void*)heat_step_kernel<ST, BC, false>;
    if (variant == GS_KERNEL_TILE && depth > 1)
        return is3d ? pick_temporal<ST, BC, true>(depth) : pick_temporal<ST, BC, false>(depth);
    return nullptr;
}

template <typename ST>
const void* pick_bc(gs_bc bc, bool is3d, int depth, int variant, int nz, int rows) {
    return bc == GS_BC_CLAMP ? pick<ST, GS_BC_CLAMP>(is3d, depth, variant, nz, rows)
                             : pick<ST, GS_BC_DIRICHLET0>(is3d, depth, variant, nz, rows);
}

int vec_elems(gs_dtype dt) { return dt == GS_F32 ? 4 : 8; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the CUDA runtime).
using PfnEncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
PfnEncodeTiled encode_tiled() {
    static const PfnEncodeTiled fn = []() -> PfnEncodeTiled {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PfnEncodeTiled>(p);
    }();
    return fn;
}

// The STREAM kernel's launch: W compute warps (block_x 512: 16, else 8),
// the tensor map of a.Tin (the grid's nx x ny x nz elements with its pitch;
// reads outside them are filled with zeros), one box a plane.
template <typename ST>
cudaError_t stream_desc(gs_bc bc, const HeatArgs& a, int block_x, CUtensorMapDataType dtype, LaunchDesc* out) {
    const int W = block_x >= 512 ? 16 : 8;
    if (a.tile_y < 1 || a.nz < 1) return cudaErrorInvalidValue;
    PfnEncodeTiled enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    StreamArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.a = a;
    const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)a.pitch * sizeof(ST), (cuuint64_t)a.plane * sizeof(ST)};
    const cuuint32_t box[3] = {(cuuint32_t)stream_cols<ST>(), (cuuint32_t)(W * kStreamRows + 2), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&sa.map, dtype, 3, const_cast<void*>(a.Tin), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const bool cl = (bc == GS_BC_CLAMP);
    const void* f = W == 16 ? (cl ? (const void*)heat_stream2_kernel<ST, GS_BC_CLAMP, 16>
                                  : (const void*)heat_stream2_kernel<ST, GS_BC_DIRICHLET0, 16>)
                            : (cl ? (const void*)heat_stream2_kernel<ST, GS_BC_CLAMP, 8>
                                  : (const void*)heat_stream2_kernel<ST, GS_BC_DIRICHLET0, 8>);
    out->func = f;
    const int ts = W * kStreamRows - 2;  // stored rows of a block
    out->block = dim3(32, W + 1, 1);
    out->grid = dim3((a.nx + kStreamTileX - 1) / kStreamTileX, (a.ny + ts - 1) / ts,
                     (a.nz + a.tile_y - 1) / a.tile_y);
    out->smem = stream_smem<ST>(W);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e != cudaSuccess) return e;
    out->set_args(sa);
    return cudaSuccess;
}

}  // namespace

size_t heat_stream_smem(gs_dtype dt, int block_x) {
    const int W = block_x >= 512 ? 16 : 8;
    return dt == GS_F32 ? stream_smem<float>(W) : stream_smem<__half>(W);
}

unsigned heat_stream_timeouts_take() {
    unsigned n = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&n, g_stream_timeouts, sizeof(n)) != cudaSuccess) return ~0u;
    cudaMemcpyToSymbol(g_stream_timeouts, &zero, sizeof(zero));
    return n;
}

cudaError_t heat_desc(gs_kind kind, gs_dtype dt, gs_bc bc, const HeatArgs& a, int block_x, int depth, int variant,
                      LaunchDesc* out) {
    const bool is3d = (kind == GS_HEAT3D);
    if (variant == GS_KERNEL_STREAM) {
        if (!is3d || depth != 2) return cudaErrorInvalidValue;
        switch (dt) {
            case GS_F32: return stream_desc<float>(bc, a, block_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, out);
            case GS_BF16: return stream_desc<__nv_bfloat16>(bc, a, block_x, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, out);
            case GS_F16: return stream_desc<__half>(bc, a, block_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, out);
        }
        return cudaErrorInvalidValue;
    }
    const void* f = nullptr;
    switch (dt) {
        case GS_F32: f = pick_bc<float>(bc, is3d, depth, variant, a.nz, a.rows); break;
        case GS_BF16: f = pick_bc<__nv_bfloat16>(bc, is3d, depth, variant, a.nz, a.rows); break;
        case GS_F16: f = pick_bc<__half>(bc, is3d, depth, variant, a.nz, a.rows); break;
    }
    if (!f) return cudaErrorInvalidValue;
    out->func = f;
    const int V = vec_elems(dt);
    if (variant == GS_KERNEL_MARCH) {
        const int zb = is3d ? std::min(std::min(a.nz, 16), std::max(1, 512 / block_x)) : 1;
        out->block = dim3(block_x, zb, 1);
        out->grid = dim3((a.nx + block_x * V - 1) / (block_x * V), (a.ny + a.rows - 1) / a.rows,
                         is3d ? (a.nz + zb - 1) / zb : 1);
        out->smem = is3d ? (size_t)2 * (zb + 2) * block_x * V * sizeof(float) : 0;
    } else if (variant == GS_KERNEL_COLUMN && depth == 2 && is3d && a.nz > kColumnMaxNz) {
        const int bw = std::max(1, std::min(block_x / 32, 4));  // warps stacked in y
        if (a.tile_y < 1) return cudaErrorInvalidValue;
        out->block = dim3(32, bw, 1);
        out->grid = dim3((a.nx + 30 * kZmW - 1) / (30 * kZmW), (a.ny + kZmR * bw - 1) / (kZmR * bw),
                         (a.nz + a.tile_y - 1) / a.tile_y);
        out->smem = 0;
    } else if (variant == GS_KERNEL_COLUMN && depth > 1 && is3d) {
        if (a.nz > kColumnMaxNz) return cudaErrorInvalidValue;
        const int bw = std::max(1, std::min(block_x / 32, 8));  // warps stacked in y
        const int rt = column3_t_rows(depth, a.rows);
        out->block = dim3(32, bw, 1);
        out->grid = dim3((a.nx + (32 - 2 * depth) - 1) / (32 - 2 * depth), (a.ny + rt * bw - 1) / (rt * bw), 1);
        out->smem = 0;
    } else if (variant == GS_KERNEL_COLUMN && depth > 1) {
        const int bw = std::max(1, std::min(block_x / 32, 8));  // warps stacked in y
        const int rt = (dt == GS_F32) ? column_t_rows<float>() : column_t_rows<__half>();
        out->block = dim3(32, bw, 1);
        out->grid = dim3((a.nx + 30 * V - 1) / (30 * V), (a.ny + rt * bw - 1) / (rt * bw), 1);
        out->smem = 0;
    } else if (variant == GS_KERNEL_COLUMN) {
        const int by = std::max(1, std::min(a.rows, 8));
        const int cw = (dt == GS_F32) ? column_width<float>(is3d) : column_width<__half>(is3d);
        const int chunks = (is3d && a.nz > kColumnMaxNz) ? (a.nz + kColumnMaxNz - 1) / kColumnMaxNz : 1;
        out->block = dim3(32, by, 1);
        out->grid = dim3((a.nx + 32 * cw - 1) / (32 * cw), (a.ny + by - 1) / by, chunks);
        out->smem = 0;
    } else if (variant == GS_KERNEL_COLUMN_SMEM) {
        if (is3d && a.nz > kColumnMaxNz) return cudaErrorInvalidValue;
        const int by = std::max(1, std::min(a.rows, 8));
        out->block = dim3(32, by, 1);
        out->grid = dim3((a.nx + 32 * V - 1) / (32 * V), (a.ny + by - 1) / by, 1);
        out->smem = heat_scol_smem(is3d ? kColumnMaxNz : 1, by, V);
    } else if (variant == GS_KERNEL_WAVE) {
        if (is3d && a.nz > kWaveMaxNz) return cudaErrorInvalidValue;
        const int stride = 30 * V;
        const int wb = is3d ? a.nz : std::max(1, block_x / 32);
        out->block = dim3(32, wb, 1);
        const int ry = is3d ? a.rows : a.rows * wb;
        out->grid = dim3((a.nx + stride - 1) / stride, (a.ny + ry - 1) / ry, 1);
        out->smem = heat_wave_smem(is3d ? a.nz : 0, depth, V);
    } else {
        out->block = dim3(block_x, 1, 1);
        out->grid = dim3((a.nx + a.tile_x - 1) / a.tile_x, (a.ny + a.tile_y - 1) / a.tile_y, 1);
        out->smem = heat_temporal_smem(is3d ? a.nz : 1, a.tile_x, a.tile_y, depth);
        if (out->smem > 227 * 1024) return cudaErrorInvalidValue;
    }
    if (out->smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
        if (e != cudaSuccess) return e;
    }
    out->set_args(a);
    return cudaSuccess;
}

GS_CHECK_UNIT(heat)

}  // namespace gs
