/*
 * graphstep — explicit iterative stencil time stepping on one GPU, with the
 * per-iteration kernels grouped into iteration batches and unrolled into CUDA
 * graphs ("Kernel Batching with CUDA Graphs", arXiv 2501.09398).
 *
 * The calls follow the paper's statement of the problem:
 *   - an iterative solver launches the same kernel(s) once per iteration
 *     (Sec. III-A, Listing 1); the launches are grouped into batches of S
 *     (Listing 2) and each batch is unrolled into a static graph built by
 *     manual graph creation: a linear chain of S kernel nodes, instantiated
 *     and uploaded before the first launch (Listing 3, "Building");
 *   - I_k iterations then take I = I_k / S graph launches (Eq. 4, Listing 3,
 *     "Launching"); iteration counts that S does not divide are handled by a
 *     peeled remainder graph (the fix the paper names in Sec. VI);
 *   - the total time is graph creation plus execution, T = T_C + T_E
 *     (Eqs. 1-6); gs_get_stats() reports the measured creation time T_C.
 *
 * Workloads (the paper's Sec. III-C applications):
 *   GS_HEAT2D  2D 5-point thermal update (Rodinia Hotspot's role);
 *   GS_HEAT3D  3D 7-point thermal update (Hotspot3D's role);
 *   GS_FDTD3D  3D Yee FDTD Maxwell solver, one H kernel and one E kernel per
 *              iteration.
 * Thermal update (per cell, FP32 arithmetic):
 *   T' = T + k*(P + cy*(T_N+T_S-2T) + cx*(T_E+T_W-2T) + cz*(t_amb-T)
 *              [+ cz2*(T_U+T_D-2T) in 3D])
 *   clamp boundary: a missing neighbour reads the cell itself (zero flux);
 *   Dirichlet-0: it reads 0.  In 3D, P is one x-y plane acting on layer 0.
 * FDTD update (normalised units, dx = 1, dt = courant number s):
 *   H -= s*curl(E) (forward differences), then E += s*curl(H) (backward
 *   differences, interior only: tangential E on the PEC walls stays 0), then
 *   a soft source Ez[src] += amp*exp(-((n - delay)/width)^2) at step n.
 *
 * Conventions for every call:
 *   - Every function returns gs_status; GS_OK is 0.  Nothing throws or aborts
 *     across the boundary.  On failure, gs_last_error(ctx) holds a message.
 *   - Device memory for fields is owned by the caller (e.g. allocated with
 *     PyTorch) and borrowed by the context; it must stay valid while bound.
 *     The context owns its graphs, its stream (only if it created one) and
 *     small scratch buffers (FDTD step counter, conversion staging).
 *   - Layout: x fastest, then y, then z.  A row holds `pitch` elements,
 *     pitch >= row width and a multiple of 16 bytes (4 f32 or 8 bf16/f16
 *     elements); the base pointer is 16-byte aligned; planes are pitch*rows
 *     elements apart.  gs_required_pitch() returns the smallest valid pitch.
 *   - All GPU work is asynchronous on the context's stream unless a call says
 *     it synchronises.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef GRAPHSTEP_H
#define GRAPHSTEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* bad handle, size, pointer, alignment or value */
    GS_ERR_CUDA = 2,        /* a CUDA runtime call failed; see gs_last_error */
    GS_ERR_OOM = 3,         /* a host or device allocation failed */
    GS_ERR_STATE = 4,       /* call not valid in the current state (e.g. unbound field) */
    GS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    GS_ERR_NUMERIC = 6,     /* non-finite values where finite ones are required */
    GS_ERR_UNSUPPORTED = 7  /* valid request the library does not provide (e.g. plan too large) */
} gs_status;

/* GS_SKELETON is the paper's skeleton application (Sec. III-C): a vector of
 * nx elements multiplied in place by a constant c, one kernel per iteration
 * (ny = nz = 1; field GS_FIELD_X; gs_set_scale sets c, default 1). */
typedef enum gs_kind { GS_HEAT2D = 0, GS_HEAT3D = 1, GS_FDTD3D = 2, GS_SKELETON = 3 } gs_kind;

/* Storage type of the fields.  Arithmetic is always FP32. */
typedef enum gs_dtype { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

/* Boundary rule.  Thermal: CLAMP or DIRICHLET0.  FDTD: PEC only. */
typedef enum gs_bc { GS_BC_CLAMP = 0, GS_BC_DIRICHLET0 = 1, GS_BC_PEC = 2 } gs_bc;

typedef enum gs_field {
    GS_FIELD_T0 = 0, /* thermal ping-pong buffer 0 (nz*ny rows of pitch) */
    GS_FIELD_T1 = 1, /* thermal ping-pong buffer 1 */
    GS_FIELD_P = 2,  /* thermal power map: one ny-row plane (layer 0 in 3D) */
    GS_FIELD_EX = 3, /* FDTD components: (N+1)*(N+1) rows of pitch each */
    GS_FIELD_EY = 4,
    GS_FIELD_EZ = 5,
    GS_FIELD_HX = 6,
    GS_FIELD_HY = 7,
    GS_FIELD_HZ = 8,
    GS_FIELD_T = 9,  /* alias: whichever of T0/T1 holds the current state */
    GS_FIELD_X = 10, /* skeleton vector: one row of nx elements */
    GS_FIELD_MAT = 11 /* FDTD material map: uint8 ids, (N+1)*(N+1) rows with
                         the same pitch (in elements) as the six components;
                         read only while a media table is set */
} gs_field;

typedef struct gs_ctx gs_ctx;

typedef struct gs_heat_coeffs {
    float k, cx, cy, cz, cz2, t_amb;
} gs_heat_coeffs;

typedef struct gs_fdtd_params {
    float courant;   /* s = c*dt/dx; stable for s < 1/sqrt(3) */
    int32_t src_on;  /* 1: soft Ez source after each E update */
    int64_t src_i, src_j, src_k;
    float src_amp, src_delay, src_width; /* amp*exp(-((n-delay)/width)^2) */
} gs_fdtd_params;

/* One row of an FDTD media table: relative permittivity, conductivity,
 * relative permeability and magnetic conductivity, in the normalised units
 * of the FDTD context (eps0 = mu0 = c = 1, dx = 1, dt = courant).  With
 * a_e = sigma*s/(2 eps_r), a_h = sigma_m*s/(2 mu_r), each step is the
 * textbook lossy-medium Yee update
 *   H <- da*H - db*curl(E),  da = (1 - a_h)/(1 + a_h), db = (s/mu_r)/(1 + a_h)
 *   E <- ca*E + cb*curl(H),  ca = (1 - a_e)/(1 + a_e), cb = (s/eps_r)/(1 + a_e)
 * (coefficients computed in double, stored as float). */
typedef struct gs_medium {
    float eps_r, sigma, mu_r, sigma_m;
} gs_medium;

#define GS_MAX_MEDIA 256

/* Thermal kernel variants (gs_plan.kernel).
 *   MARCH  depth 1 only: each thread marches a vector of cells down `rows`
 *          rows; any nz.
 *   WAVE   depth 1, 2 or 4, 2D or nz <= 16: each warp marches `rows` rows and
 *          advances `temporal_depth` time levels in one pass (register
 *          windows per level; block_x/32 warps per block in 2D, one warp
 *          per plane in 3D).
 *   TILE   depth 2 or 4: overlapped shared-memory tile of tile_x x tile_y
 *          columns (all nz planes) with a t-wide halo.
 *   COLUMN depth 1: each thread owns one vector of cells at one y with
 *          every plane of its column in registers (no march, no shared
 *          memory); stacks of more than 8 planes in chunks of 8 (the planes
 *          just below and above a chunk loaded as halos); `rows` (<= 8) warps
 *          per block stacked in y.  Depth 2 or 4 in 2D: each thread owns
 *          one vector of cells in 4 rows (2 for bf16/f16), loads those rows
 *          and 2t halo rows at once and advances t levels in registers
 *          (lanes 0 and 31 of a warp are halo lanes); block_x/32 warps per
 *          block stacked in y.  Depth 2 or 4 in 3D with nz <= 8: each lane
 *          owns one cell at R rows (R = 4, or 2 with rows = 2, at depth 2; 2
 *          at depth 4) of every plane, t lanes at each warp end are halo
 *          lanes; block_x/32 warps per block.  Depth 2 in 3D with nz > 8:
 *          blocks march tile_y planes in z (default 32), two cells a lane,
 *          four rows a warp, min(block_x/32, 4) warps a block.
 *   COLUMN_SMEM  as COLUMN, but each thread loads only its own row of every
 *          plane; rows y-1 / y+1 come from shared memory after one barrier
 *          (fewer registers and L2 requests).
 *   STREAM 3D at depth 2 only: a block marches tile_y planes in z over an
 *          x-y tile of 128 x (2W - 2) cells (W = 16 compute warps with
 *          block_x = 512, 8 with block_x = 256; block_x must be one of the
 *          two), each lane four cells at two rows, its level-0 planes
 *          arriving in shared memory through the Tensor Memory Accelerator
 *          (a ring of six plane stages), level 1 of each plane kept in
 *          shared memory for its neighbours.  Any nz.
 *   AUTO   depth 1, 2D, and 3D with nz <= 8: COLUMN; other 3D stacks at
 *          depth 2: WAVE for nz <= 16, else STREAM (block_x 256 unless 256
 *          or 512 is given; with another block_x, COLUMN's z march); at
 *          depth 4: WAVE for nz <= 16, else TILE.
 * FDTD variants: COLUMN (default) and MARCH run the two launches of a step
 * (H, then E).  FUSED runs one launch a step, out of place into a second set
 * of the six components that the context allocates (steps in pairs, so the
 * state ends in the bound fields; an odd last step runs as the two
 * launches), bit-identical to the two launches: with tile_y = 0 a thread
 * owns four cells along i at one (j, k) and recomputes the H values of rows
 * j-1 and planes k-1 that its E update reads; with tile_y >= 1 a block of
 * 32 x rows threads marches tile_y planes in k and keeps H of the plane
 * below in registers (only row j-1 is recomputed). */
typedef enum gs_kernel {
    GS_KERNEL_AUTO = 0,
    GS_KERNEL_MARCH = 1,
    GS_KERNEL_WAVE = 2,
    GS_KERNEL_TILE = 3,
    GS_KERNEL_COLUMN = 4,
    GS_KERNEL_COLUMN_SMEM = 5,
    GS_KERNEL_FUSED = 6,
    GS_KERNEL_STREAM = 7
} gs_kernel;

/* Block traversal order of consecutive launches (gs_plan.traverse,
 * gs_multi_plan.traverse).  ALTERNATE walks the grid's blocks in reverse on
 * every other launch (thermal: launches that read T1; FDTD: the E half-step;
 * instance batches: launches that read T1), so a step starts on the rows the
 * previous step touched last, which are still in L2 when the working set is
 * a little larger than L2 (measured on GB300: 2D 3072^2 +21 %, 4096^2 +12 %;
 * none for an L2-resident field).  The order of blocks never changes a
 * result.  AUTO: ALTERNATE when the bytes one step touches exceed half of
 * the L2 cache, else FORWARD.  No counterpart in the paper (a scheduling
 * detail of the stepping kernels). */
typedef enum gs_traverse { GS_TRAVERSE_AUTO = 0, GS_TRAVERSE_FORWARD = 1, GS_TRAVERSE_ALTERNATE = 2 } gs_traverse;

/* Launch plan.  Zero fields select defaults.
 *   block_x        threads along x per block (multiple of 32; <= 512 thermal,
 *                  <= 256 FDTD)
 *   rows           MARCH / WAVE: rows each block (or warp) marches along y;
 *                  COLUMN at depth 1: warps per block stacked in y (more
 *                  than 8 act as 8; at depth 2/4 block_x/32 warps); FDTD
 *                  COLUMN: j rows per block; FDTD MARCH: k planes per block
 *   tile_x, tile_y output tile of the TILE kernel; tile_y is also the z
 *                  chunk a block marches in the depth-2 COLUMN kernel of
 *                  stacks deeper than 8 planes and in the STREAM kernel, and
 *                  the k planes a block marches in the FDTD FUSED kernel (0:
 *                  no march; range [0, 2^20])
 *   temporal_depth thermal steps fused in one launch: 1, 2 or 4; a depth-t
 *                  launch is bit-identical to t depth-1 launches
 *   use_pdl        1: graph nodes (and per-step launches) use programmatic
 *                  dependent launch, so the next kernel's launch overlaps the
 *                  tail of the previous one; results are unchanged
 *   device_launch  1: instantiate graphs with cudaGraphInstantiateFlagDeviceLaunch
 *                  as in the paper's Listing 3 (not combinable with use_pdl) */
typedef struct gs_plan {
    int32_t block_x;
    int32_t rows;
    int32_t tile_x;
    int32_t tile_y;
    int32_t temporal_depth;
    int32_t use_pdl;
    int32_t device_launch;
    int32_t kernel; /* gs_kernel; FDTD: COLUMN (default: four cells along i
                       per thread, block 32 x rows x 8/rows), MARCH
                       (block_x threads marching `rows` k planes) or FUSED
                       (one launch a step; see gs_kernel) */
    int32_t graph_loop; /* 0: the floor(n/S) batches are floor(n/S) graph
                           launches (Listing 3).  1: one launch of a graph
                           whose conditional while node repeats the batch on
                           the device (Sec. V's conditional nodes): a small
                           kernel at the end of each trip counts the trips
                           down and clears the condition after the last; when
                           a batch flips the buffer parity the loop body is
                           two batches and an odd last batch runs as a plain
                           batch graph.  Same results bit for bit.  Not with
                           device_launch (a device-launch graph holds no
                           conditional node): GS_ERR_UNSUPPORTED. */
    int32_t traverse;   /* gs_traverse (0: AUTO); ignored by the skeleton kernel */
} gs_plan;

typedef struct gs_stats {
    double last_build_seconds;  /* host wall time of the last graph build:
                                   create + add nodes + instantiate + upload
                                   (the paper's T_C, Eq. 2, incl. upload) */
    int64_t last_build_nodes;   /* kernel nodes in that graph */
    int64_t graphs_built;       /* executable graphs built since creation */
    int64_t graph_launches;     /* cudaGraphLaunch calls issued */
    int64_t kernel_launches;    /* direct kernel launches issued */
    int64_t iterations;         /* iterations issued (thermal steps / FDTD H+E pairs) */
} gs_stats;

/* ------------------------------------------------------------- basics -- */

/* Library version as major*10000 + minor*100 + patch. */
int gs_version(void);

/* Static, human-readable name of a status code (never NULL). */
const char *gs_status_string(gs_status s);

/* Message of the last failed call on ctx ("" if none).  The pointer stays
 * valid until the next call on ctx.  ctx == NULL gives the message of the
 * last call on this thread that failed with no context to hold it: a failed
 * gs_create or gs_multi_create, a NULL handle, and the host-only calls
 * (gs_required_pitch, gs_model_*, gs_features, gs_plan_check,
 * gs_candidates, argument errors of gs_pick and gs_multi_step_noalloc).
 * A successful call does not clear it. */
const char *gs_last_error(const gs_ctx *ctx);

/* Smallest valid row pitch (elements) for rows of `width` elements of
 * `dtype`: width rounded up to a multiple of 16 bytes.
 * Errors: GS_ERR_INVALID_ARG for width < 1 or an unknown dtype. */
gs_status gs_required_pitch(gs_dtype dtype, int64_t width, int64_t *pitch_out);

/* ------------------------------------------------------ context set-up -- */

/* Create a stepping context.
 *   kind     GS_HEAT2D (nz must be 1), GS_HEAT3D, GS_FDTD3D (nx == ny == nz
 *            == N cells; each component is an (N+1)^3 array), GS_SKELETON
 *            (ny == nz == 1; nx elements, up to 2^31)
 *   nx,ny,nz grid size in cells, each in [1, 2^20], total < 2^31 elements
 *   storage  field storage type
 *   bc       GS_BC_CLAMP / GS_BC_DIRICHLET0 (thermal), GS_BC_PEC (FDTD);
 *            ignored for GS_SKELETON
 *   stream   cudaStream_t to run on, borrowed (cudaStreamLegacy and
 *            cudaStreamPerThread are accepted); NULL: the context creates
 *            (and later destroys) its own non-blocking stream, as the
 *            paper's Listing 3 does.
 * Defaults: thermal coefficients k=0.5, cx=cy=0.1, cz=0.01, cz2=0.05,
 * t_amb=80; FDTD courant 0.5, source off; plan defaults, depth 1, no PDL.
 * The CUDA device current on the calling thread is used.
 * Errors: GS_ERR_INVALID_ARG (sizes, kind/bc mismatch), GS_ERR_CUDA,
 * GS_ERR_OOM.  *out is NULL on failure. */
gs_status gs_create(gs_ctx **out, gs_kind kind, int64_t nx, int64_t ny, int64_t nz,
                    gs_dtype storage, gs_bc bc, void *stream);

/* Destroy ctx: synchronises its stream, frees graphs and scratch, destroys
 * the stream if the context created it.  Bound field memory is untouched.
 * NULL is accepted (no-op). */
gs_status gs_destroy(gs_ctx *ctx);

/* Replace the thermal coefficients (GS_HEAT2D / GS_HEAT3D only).  Built
 * graphs are discarded (their nodes hold the old values).  Non-finite
 * values give GS_ERR_NUMERIC. */
gs_status gs_set_heat_coeffs(gs_ctx *ctx, const gs_heat_coeffs *c);

/* Replace the FDTD parameters (GS_FDTD3D only).  The source cell must lie
 * inside the (N+1)^3 arrays.  Built graphs are discarded. */
gs_status gs_set_fdtd_params(gs_ctx *ctx, const gs_fdtd_params *p);

/* FDTD in linear, possibly lossy media (an extension of the paper's vacuum
 * cavity solver, Sec. III-C): every component at element offset c takes
 * the material GS_FIELD_MAT[c] (the cell whose lower corner is its index
 * (i, j, k)); ids >= n are vacuum.  n = 0 returns to vacuum (the map is
 * then not read).  Rows need finite eps_r > 0, mu_r > 0, sigma >= 0,
 * sigma_m >= 0 (else GS_ERR_INVALID_ARG / GS_ERR_NUMERIC); n > 256 gives
 * GS_ERR_INVALID_ARG.  Stepping with a table needs the map bound
 * (GS_ERR_STATE) and the COLUMN kernels or the FUSED march (plan.tile_y
 * >= 1); GS_ERR_UNSUPPORTED for MARCH and for FUSED with tile_y = 0.
 * The table is copied; built graphs are discarded. */
gs_status gs_set_fdtd_media(gs_ctx *ctx, const gs_medium *table, int32_t n);

/* The skeleton application's constant c (GS_SKELETON only); non-finite c
 * gives GS_ERR_NUMERIC.  Built graphs are discarded. */
gs_status gs_set_scale(gs_ctx *ctx, float c);

/* Replace the launch plan (see gs_plan).  Zero fields take defaults.  A plan
 * the kernels cannot run on this grid (shared-memory tile too large,
 * temporal depth on FDTD, bad block size) gives GS_ERR_UNSUPPORTED or
 * GS_ERR_INVALID_ARG and leaves the old plan in place.  Built graphs are
 * discarded. */
gs_status gs_set_plan(gs_ctx *ctx, const gs_plan *plan);

/* The plan in effect, with defaults filled in. */
gs_status gs_get_plan(const gs_ctx *ctx, gs_plan *out);

/* Bind caller-owned device memory to a field.
 *   ptr    device pointer, 16-byte aligned; NULL unbinds
 *   pitch  row pitch in elements (>= row width, multiple of 16 bytes)
 * The buffer must hold rows*pitch elements: ny rows (2D, and P), nz*ny
 * rows (3D thermal), (N+1)^2 rows of N+1 used elements (each FDTD
 * component).  GS_FIELD_T binds the buffer that currently holds the state.
 * Rebinding discards built graphs. */
gs_status gs_bind_field(gs_ctx *ctx, gs_field id, void *ptr, int64_t pitch);

/* Copy a dense float32 host array (x fastest, no padding) into a bound
 * field, rounding to the storage type (round to nearest even).  n must be
 * the field's dense element count.  Synchronises the context stream before
 * returning, so the host buffer may be reused at once. */
gs_status gs_upload(gs_ctx *ctx, gs_field id, const float *host, int64_t n);

/* Copy a dense uint8 host array ((N+1)^3 ids, i fastest) into the bound
 * GS_FIELD_MAT of an FDTD context.  Synchronous. */
gs_status gs_upload_u8(gs_ctx *ctx, gs_field id, const uint8_t *host, int64_t n);

/* Copy a bound field into a dense float32 host array (widened from the
 * storage type).  n must be the field's dense element count.  Synchronises
 * the context stream (all queued steps finish first). */
gs_status gs_read_field(gs_ctx *ctx, gs_field id, float *host_out, int64_t n);

/* Which thermal buffer (0 or 1) holds the current state. */
gs_status gs_get_parity(const gs_ctx *ctx, int32_t *parity_out);

/* Declare which thermal buffer (0 or 1) holds the current state. */
gs_status gs_set_parity(gs_ctx *ctx, int32_t parity);

/* FDTD time index n of the next step (the source uses it).  gs_set_time
 * writes it to the device counter on the context stream; it is ordered with
 * the steps around it.  Thermal contexts only keep the host count. */
gs_status gs_set_time(gs_ctx *ctx, int64_t n);
gs_status gs_get_time(const gs_ctx *ctx, int64_t *n_out);

/* ------------------------------------------------------------ stepping -- */

/* Advance n_iters iterations (thermal steps, or FDTD H+E pairs).
 *   batch_size == 0  per-step launches: one kernel launch per iteration
 *                    (per fused group of temporal_depth iterations) — the
 *                    paper's baseline, Listing 1;
 *   batch_size  > 0  iteration batching: floor(n/S) launches of a graph of
 *                    S iterations (Listing 3), then one launch of a cached
 *                    remainder graph of n mod S iterations (loop peeling).
 *                    Graphs are built on first use and cached per
 *                    (S, buffer parity); two exec graphs exist when a batch
 *                    flips the ping-pong parity.
 * Results are bit-identical for every batch_size, temporal depth and PDL
 * setting.  Asynchronous.  Errors: GS_ERR_STATE if a required field is
 * unbound; GS_ERR_INVALID_ARG for n_iters < 0 or batch_size < 0. */
gs_status gs_step(gs_ctx *ctx, int64_t n_iters, int64_t batch_size);

/* Build, instantiate and upload the graph(s) for batches of S iterations
 * starting from the current parity (and the other parity when S flips it),
 * synchronously, timing the host wall clock into gs_stats.last_build_seconds.
 * Replaces earlier graphs of the same S. */
gs_status gs_graph_build(gs_ctx *ctx, int64_t batch_size);

/* Launch the graph built by the last gs_graph_build n_launches times
 * (S*n_launches iterations).  Asynchronous.  GS_ERR_STATE if none is built. */
gs_status gs_graph_launch(gs_ctx *ctx, int64_t n_launches);

/* Destroy every cached graph of ctx. */
gs_status gs_graph_destroy(gs_ctx *ctx);

/* Wait for all work queued on the context stream. */
gs_status gs_sync(gs_ctx *ctx);

/* Counters and the last measured graph build time. */
gs_status gs_get_stats(const gs_ctx *ctx, gs_stats *out);

/* ------------------------------------------------------------ autotuner -- */

typedef struct gs_tune_candidate {
    gs_plan plan;        /* launch plan (zero fields: defaults) */
    int64_t batch_size;  /* iteration batch size S; 0 = per-step launches */
} gs_tune_candidate;

typedef struct gs_tune_result {
    gs_plan plan;             /* the plan as applied (defaults filled in) */
    int64_t batch_size;
    double build_seconds;     /* T_C: gs_graph_build host wall time (0 for S = 0) */
    double exec_ms_per_iter;  /* T_E / n_iters, best of `reps` runs, CUDA events
                                 on the context stream, graphs cached */
    double total_ms;          /* build_seconds*1e3 + T_E of one n_iters run:
                                 the paper's T = T_C + T_E (Eq. 1) */
    int32_t status;           /* GS_OK, or why the candidate was skipped
                                 (e.g. GS_ERR_UNSUPPORTED for a plan that does
                                 not fit this grid) */
    int32_t reserved;
} gs_tune_result;

/* Time every candidate on the context's own bound fields: set its plan,
 * build its graphs (timed: T_C), run n_iters iterations once to warm up,
 * then `reps` timed runs of n_iters iterations.  results[i] describes
 * cands[i]; *best_index (may be NULL) receives the index with the smallest
 * total_ms, the candidate that minimises T = T_C + T_E for a run of n_iters
 * iterations (the paper's selection of the iteration batch size, Sec. III-B,
 * extended to the launch plan).  The fields, buffer parity, time counter and
 * plan are restored afterwards (the fields are snapshotted into temporary
 * device memory first).  Synchronous.  Errors: GS_ERR_INVALID_ARG,
 * GS_ERR_STATE (unbound fields), GS_ERR_CUDA, GS_ERR_OOM (snapshot),
 * GS_ERR_UNSUPPORTED if no candidate could run. */
gs_status gs_autotune(gs_ctx *ctx, int64_t n_iters, int32_t reps, const gs_tune_candidate *cands, int32_t n_cands,
                      gs_tune_result *results, int32_t *best_index);

/* ------------------------------------------------------ analytic model -- */

/* The paper's performance model (Sec. III-B): T = T_C + T_E (Eq. 1),
 * T_C = k_c*S + b_c (Eq. 2), T_E = a/S + b (Eq. 6, from Eqs. 3-5 with
 * a = I_k(T_a - T_i), b = I_k(T_k + T_i) - T_a + T_l), all in seconds for a
 * run of I_k iterations.  mae_* are the fits' mean absolute errors (the
 * paper's Table I reports the same quantities). */
typedef struct gs_model {
    double k_c, b_c;  /* Eq. 2 */
    double a, b;      /* Eq. 6 */
    double mae_create, mae_exec;
} gs_model;

/* Least-squares fit of Eq. 2 to (S[i], t_create[i]) and of Eq. 6 to
 * (S[i], t_exec[i]), n >= 2 points with at least two distinct S >= 1.
 * Host only (no GPU needed).  Errors: GS_ERR_INVALID_ARG, GS_ERR_NUMERIC;
 * message in gs_last_error(NULL). */
gs_status gs_model_fit(const double *S, const double *t_create, const double *t_exec, int32_t n, gs_model *out);

/* Eq. 1 for batch size S >= 1: k_c*S + b_c + a/S + b. */
gs_status gs_model_total(const gs_model *m, double S, double *total_out);

/* The batch size among cands[0..n) (each >= 1, e.g. the divisors of I_k the
 * paper admits, Sec. III-B) that minimises Eq. 1; ties go to the smaller S.
 * *best_T (may be NULL) receives the model's total. */
gs_status gs_model_pick(const gs_model *m, const int64_t *cands, int32_t n, int64_t *best_S, double *best_T);

/* Measure T_C and T_E on the context for each S in S_list (runs of n_iters
 * iterations with the context's current plan, via gs_autotune, so the fields
 * are restored) and fit the model.  Choose S values that divide n_iters so
 * that T_E holds no remainder graph. */
gs_status gs_model_calibrate(gs_ctx *ctx, int64_t n_iters, const int64_t *S_list, int32_t n, int32_t reps,
                             gs_model *out);

/* ------------------------------------------------- learned cost model -- */

/* A small MLP that predicts log(milliseconds per iteration) of running a
 * workload with a candidate (launch plan, batch size S), trained on timings
 * the library sweeps itself (gs_autotune), used to pick the candidate with
 * the smallest prediction.  This takes the place of the paper's analytic
 * model (Sec. III-B) in choosing S, and extends the choice to the launch
 * plan and temporal depth — the automatic characterisation and batch-size
 * selection the paper leaves as future work (Sec. VI).
 * Network: GS_MLP_INPUTS -> GS_MLP_HIDDEN -> GS_MLP_HIDDEN -> 1, ReLU, one
 * flat FP32 parameter array: W1[32][18] | b1[32] | W2[32][32] | b2[32] |
 * W3[32] | b3.  Inputs are standardised inside the kernels with a stored
 * per-feature mean and 1/std.  Loss: mean squared error.  Training: Adam
 * (0.9, 0.999, 1e-8), minibatches in row order; one epoch is replayed as a
 * CUDA graph.  All arrays passed as X / y are device memory, X row-major
 * [n_rows][GS_MLP_INPUTS] float32, y [n_rows] float32. */
#define GS_MLP_INPUTS 18
#define GS_MLP_HIDDEN 32
#define GS_MLP_PARAMS 1697

typedef struct gs_mlp gs_mlp;

/* Describes a stepping problem for the feature vector. */
typedef struct gs_workload {
    int32_t kind;     /* gs_kind */
    int32_t dtype;    /* gs_dtype */
    int64_t nx, ny, nz;
    int64_t n_iters;  /* iterations of the run (the paper's I_k) */
} gs_workload;

/* Feature vectors (n x GS_MLP_INPUTS floats, host memory) of a workload
 * with each candidate: log2 nx, log2 ny, log2 nz, one-hot kind (3), kernels
 * per iteration (FDTD: 2, or 1 for the FUSED kernel; thermal 1), log2 n_iters, one-hot dtype (3), log2 S (0 for S = 0),
 * [S == 0], log2 block_x, log2 rows, temporal depth, [kernel is COLUMN or
 * COLUMN_SMEM], [kernel is COLUMN_SMEM] (GS_KERNEL_AUTO resolved as
 * gs_set_plan does).  Candidates must give block_x, rows and
 * temporal_depth explicitly.  Host only. */
gs_status gs_features(const gs_workload *w, const gs_tune_candidate *c, int32_t n, float *out);

/* Create a model with Glorot-uniform weights drawn from splitmix64(seed),
 * zero biases, identity normalisation, on `stream` (NULL: own stream). */
gs_status gs_mlp_create(gs_mlp **out, uint64_t seed, void *stream);
gs_status gs_mlp_destroy(gs_mlp *m);
const char *gs_mlp_last_error(const gs_mlp *m);

/* Parameters (GS_MLP_PARAMS floats, host).  Setting them resets Adam. */
gs_status gs_mlp_set_params(gs_mlp *m, const float *host, int64_t n);
gs_status gs_mlp_get_params(gs_mlp *m, float *host, int64_t n);

/* Feature standardisation: fit mean and 1/std (population) of X's columns
 * on the GPU, or set / get them (GS_MLP_INPUTS floats each, host). */
gs_status gs_mlp_fit_normalization(gs_mlp *m, const float *X, int64_t n_rows);
gs_status gs_mlp_set_normalization(gs_mlp *m, const float *mean, const float *inv_std);
gs_status gs_mlp_get_normalization(gs_mlp *m, float *mean, float *inv_std);

/* Mean squared error over the rows and its gradient with respect to the
 * parameters (grad_host: GS_MLP_PARAMS floats or NULL).  Synchronous. */
gs_status gs_mlp_loss_grad(gs_mlp *m, const float *X, const float *y, int64_t n_rows, float *loss_out,
                           float *grad_host);

/* `epochs` passes of Adam over minibatches of batch_rows rows at learning
 * rate lr; *final_loss (may be NULL) gets the loss over all rows after
 * training.  Synchronous. */
gs_status gs_mlp_train(gs_mlp *m, const float *X, const float *y, int64_t n_rows, int32_t epochs, int32_t batch_rows,
                       float lr, float *final_loss);

/* Predictions for n_rows rows into device memory `pred`.  Asynchronous. */
gs_status gs_mlp_predict(gs_mlp *m, const float *X, int64_t n_rows, float *pred);

/* The row with the smallest prediction (ties: lowest row) and its value.
 * Synchronous. */
gs_status gs_mlp_argmin(gs_mlp *m, const float *X, int64_t n_rows, int64_t *best_row, float *best_pred);

/* As gs_mlp_argmin for an ensemble of k models: the row with the smallest
 * mean prediction of models[0..k-1] (each with its own normalisation), and
 * that mean.  Runs on models[0]'s stream after waiting for the others'.
 * Synchronous.  Errors are reported through gs_mlp_last_error(models[0])
 * for CUDA failures, gs_last_error(NULL) for bad arguments. */
gs_status gs_mlp_argmin_ensemble(gs_mlp *const *models, int32_t k, const float *X, int64_t n_rows,
                                 int64_t *best_row, float *best_pred);

/* ------------------------------- choosing the plan and the batch size -- */

/* Would gs_set_plan accept `plan` on a context of workload w (kind, dtype,
 * nx, ny, nz; n_iters is not read)?  The same checks, on the host, without a
 * context or a GPU.  resolved (may be NULL) receives the plan with defaults
 * filled in and GS_KERNEL_AUTO resolved.  Errors: as gs_set_plan
 * (GS_ERR_INVALID_ARG, GS_ERR_UNSUPPORTED), and GS_ERR_INVALID_ARG for a
 * workload gs_create would refuse; message in gs_last_error(NULL). */
gs_status gs_plan_check(const gs_workload *w, const gs_plan *plan, gs_plan *resolved);

/* The candidate (launch plan, batch size) pairs the pickers choose from for
 * a thermal or FDTD workload: each of the workload's candidate plans (the
 * library's default plan among them) with batch size 0 (per-step launches)
 * and the paper's swept graph batch sizes 1, 10, 50, 100, 500, 1000
 * (Sec. IV), plan after plan.  Plans carry block_x, rows, temporal_depth,
 * kernel and tile_y (the FDTD FUSED march's planes a block; 0 elsewhere);
 * their other fields are 0.  Some plans may not fit the grid
 * (see gs_plan_check).  out == NULL (capacity 0) only counts: *n_out gets
 * the number.  Host only.  Errors: GS_ERR_INVALID_ARG (bad workload kind,
 * or capacity below the count, with *n_out set). */
gs_status gs_candidates(const gs_workload *w, gs_tune_candidate *out, int32_t capacity, int32_t *n_out);

/* The learned choice (the automatic batch-size selection the paper leaves
 * to future work, Sec. VI, widened to the launch plan and temporal depth):
 * among the workload's candidates that fit its grid, the one the ensemble
 * models[0..k-1] predicts fastest for a run of w->n_iters iterations
 * (gs_features, then gs_mlp_argmin_ensemble); nothing of the workload runs.
 * *pred_ms_per_iter (may be NULL) gets the predicted milliseconds per
 * iteration with graph creation amortised over the run.  Synchronous (on
 * models[0]'s stream).  Errors: GS_ERR_INVALID_ARG, GS_ERR_UNSUPPORTED (no
 * candidate fits), GS_ERR_NUMERIC (no finite prediction), GS_ERR_CUDA /
 * GS_ERR_OOM (message in gs_mlp_last_error(models[0])).  The exhaustive
 * fallback (and the yardstick of a pick's regret) is gs_autotune over the
 * same gs_candidates on a context of the workload. */
gs_status gs_pick(gs_mlp *const *models, int32_t k, const gs_workload *w, gs_tune_candidate *best,
                  float *pred_ms_per_iter);

/* The trained ensemble compiled into the library: GS_MLP_BUILTIN_MEMBERS
 * models trained with the library's own kernels on the GB300 sweep the
 * package ships (gs_mlp_builtin_info() names the sweep, epochs and losses).
 * gs_mlp_create_builtin creates member `member` (weights and normalisation
 * set) on `stream` (NULL: its own).  Errors: GS_ERR_INVALID_ARG (member out
 * of range), GS_ERR_UNSUPPORTED (a build without a trained ensemble), and
 * those of gs_mlp_create; message in gs_last_error(NULL). */
#define GS_MLP_BUILTIN_MEMBERS 3
gs_status gs_mlp_create_builtin(gs_mlp **out, int32_t member, void *stream);
const char *gs_mlp_builtin_info(void);

/* The learned choice for a context, with the library's own ensemble: the
 * candidate (plan, batch size) gs_pick chooses for a run of n_iters
 * iterations of ctx's workload (kind, storage type, grid) with the
 * compiled-in models, applied with gs_set_plan (the candidate's block_x,
 * rows, temporal_depth, kernel and tile_y; its other plan fields 0); on an
 * FDTD context with a media table only the plans media run on (COLUMN and
 * the FUSED march) are considered.  *plan_out (may
 * be NULL) receives the applied plan, *batch_out the batch size to pass to
 * gs_step (0: per-step launches), *pred_ms_per_iter (may be NULL) the
 * prediction.  Runs nothing of the workload.  Synchronous (on ctx's stream).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_UNSUPPORTED (skeleton contexts, a build
 * without a trained ensemble, no candidate fits), GS_ERR_NUMERIC,
 * GS_ERR_CUDA / GS_ERR_OOM; message in gs_last_error(ctx). */
gs_status gs_pick_ctx(gs_ctx *ctx, int64_t n_iters, gs_plan *plan_out, int64_t *batch_out, float *pred_ms_per_iter);

/* The paper's choice (Sec. III-B): on ctx at its current plan, measure graph
 * creation and execution for the batch sizes 1, 10, 50, 100, 500, 1000 that
 * do not exceed n_iters (gs_model_calibrate: reps timed runs of n_iters
 * iterations each, fields restored), fit Eqs. 2 and 6, and take the batch
 * size minimising Eq. 1 (gs_model_pick).  *model_out (may be NULL) gets the
 * fit.  Synchronous; runs the workload.  Errors: GS_ERR_INVALID_ARG
 * (n_iters < 10, reps < 1), and those of gs_model_calibrate. */
gs_status gs_pick_analytic(gs_ctx *ctx, int64_t n_iters, int32_t reps, int64_t *batch_out, gs_model *model_out);

/* ------------------------------------------------ uneven instance batch -- */

/* Many independent 2D thermal grids of different sizes advanced together.
 * Each instance behaves like a GS_HEAT2D context (same fields, layout and
 * update); all instances share the stream, coefficients and buffer parity.
 * This extends the paper's iteration batching (Sec. III-A) across problems:
 * one launch per iteration covers every instance, and iteration batches of
 * those launches are recorded into one graph. */
typedef struct gs_multi gs_multi;

typedef enum gs_multi_mode {
    GS_MULTI_FUSED = 0,    /* one persistent kernel per iteration over all
                              (instance, tile) work items, largest instances
                              first; batch_size > 0 records batches into a
                              graph by stream capture */
    GS_MULTI_SEPARATE = 1  /* baseline: each instance stepped by its own
                              launches (per-step, or its own graphs), one
                              instance after another on the stream; the
                              instance contexts run the depth-1 MARCH kernel
                              with the batch plan's block_x and rows */
} gs_multi_mode;

typedef struct gs_multi_plan {
    int32_t block_x; /* MARCH tiles: threads per block (multiple of 32, <= 512); default 64 */
    int32_t rows;    /* rows per work item (COLUMN: <= 8); default 8 (MARCH), 4 (COLUMN) */
    int32_t blocks;  /* persistent grid size; 0: SM count x occupancy */
    int32_t use_pdl; /* programmatic dependent launch between iterations */
    int32_t kernel;  /* work-item tile: GS_KERNEL_MARCH (default; block_x threads
                        marching `rows` rows) or GS_KERNEL_COLUMN (32 x rows
                        threads, one row per warp row) */
    int32_t traverse; /* gs_traverse (0: AUTO, on the batch's total bytes); the
                         reversed launches take the work items last to first */
    int32_t temporal_depth; /* 1 (0: default), 2 or 4 with GS_KERNEL_COLUMN:
                               each fused launch advances every instance that
                               many steps (the depth-t COLUMN tile); n mod t
                               steps run as depth-1 launches.  Results are
                               bit-identical to depth 1. */
} gs_multi_plan;

/* Create a batch of n instances, instance i of size nx[i] x ny[i] (each in
 * [1, 2^20]).  storage/bc/stream as for gs_create (the batch's stream must
 * be capturable, i.e. not the legacy default stream, for batch_size > 0 in
 * GS_MULTI_FUSED mode).  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_OOM;
 * *out is NULL on failure. */
gs_status gs_multi_create(gs_multi **out, int32_t n, const int64_t *nx, const int64_t *ny, gs_dtype storage,
                          gs_bc bc, void *stream);

/* Destroy the batch (synchronises; frees graphs, the device descriptor
 * table and the instance contexts).  NULL is accepted. */
gs_status gs_multi_destroy(gs_multi *m);

/* Message of the last failed call on m ("" if none). */
const char *gs_multi_last_error(const gs_multi *m);

/* Thermal coefficients for every instance (default as gs_create). */
gs_status gs_multi_set_heat_coeffs(gs_multi *m, const gs_heat_coeffs *c);

/* Launch plan (zero fields take defaults).  Discards built graphs. */
gs_status gs_multi_set_plan(gs_multi *m, const gs_multi_plan *p);

/* Bind caller-owned device memory to field T0, T1 or P of instance i (as
 * gs_bind_field; GS_FIELD_T is not accepted here). */
gs_status gs_multi_bind_field(gs_multi *m, int32_t i, gs_field id, void *ptr, int64_t pitch);

/* Upload / read back a field of instance i (as gs_upload / gs_read_field;
 * GS_FIELD_T is the current buffer). */
gs_status gs_multi_upload(gs_multi *m, int32_t i, gs_field id, const float *host, int64_t n);
gs_status gs_multi_read_field(gs_multi *m, int32_t i, gs_field id, float *host_out, int64_t n);

/* Advance every instance by n_iters iterations (see gs_multi_mode).  Results
 * are bit-identical across modes and batch sizes.  Asynchronous.
 * GS_ERR_STATE if a field of some instance is unbound. */
gs_status gs_multi_step(gs_multi *m, int64_t n_iters, int64_t batch_size, gs_multi_mode mode);

/* Buffer parity shared by all instances (0: T0 holds the state). */
gs_status gs_multi_get_parity(const gs_multi *m, int32_t *parity_out);

/* Wait for the batch's stream. */
gs_status gs_multi_sync(gs_multi *m);

/* Counters summed over the fused kernel and every instance context. */
gs_status gs_multi_get_stats(const gs_multi *m, gs_stats *out);

/* Autotuning an instance batch (the batch's counterpart of gs_autotune):
 * candidates are (fused-kernel plan, batch size S) pairs; S = 0 times
 * per-step fused launches. */
typedef struct gs_multi_tune_candidate {
    gs_multi_plan plan;  /* zero fields: defaults */
    int64_t batch_size;
} gs_multi_tune_candidate;

typedef struct gs_multi_tune_result {
    gs_multi_plan plan;       /* as applied (defaults filled in) */
    int64_t batch_size;
    double build_seconds;     /* T_C: host wall time of capturing, instantiating
                                 and uploading the batch graphs (0 for S = 0) */
    double exec_ms_per_iter;  /* best of `reps` timed runs, CUDA events */
    double total_ms;          /* build_seconds*1e3 + T_E of one n_iters run */
    int32_t status;           /* GS_OK, or why the candidate was skipped */
    int32_t reserved;
} gs_multi_tune_result;

/* The candidates the batch's tuner sweeps: MARCH tiles (block_x 64, 128;
 * rows 4, 8, 16), COLUMN tiles at depth 1 (rows 2, 4, 8), 2 (rows 1, 2, 4)
 * and 4 (rows 1, 2), each with S = 0, 10, 100 and 1000, plan after plan.
 * out == NULL (capacity 0) only counts.  Host only.  Errors:
 * GS_ERR_INVALID_ARG (capacity below the count, *n_out set). */
gs_status gs_multi_candidates(const gs_multi *m, gs_multi_tune_candidate *out, int32_t capacity, int32_t *n_out);

/* Time every candidate on the batch's own bound fields, fused mode: set its
 * plan, capture its batch graphs (timed: T_C), run n_iters iterations once
 * to warm up, then `reps` timed runs; results[i] describes cands[i] and
 * *best_index (may be NULL) the candidate with the smallest total_ms (the
 * paper's T = T_C + T_E, Eq. 1, for a run of n_iters iterations).  Every
 * instance's fields, the buffer parity and the plan are restored afterwards
 * (the current buffers are snapshotted into temporary device memory).
 * Synchronous.  Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE (unbound fields),
 * GS_ERR_CUDA, GS_ERR_OOM (snapshot), GS_ERR_UNSUPPORTED if no candidate
 * could run. */
gs_status gs_multi_autotune(gs_multi *m, int64_t n_iters, int32_t reps, const gs_multi_tune_candidate *cands,
                            int32_t n_cands, gs_multi_tune_result *results, int32_t *best_index);

/* The plan in effect, defaults filled in. */
gs_status gs_multi_get_plan(const gs_multi *m, gs_multi_plan *out);

/* ----------------------------------------------- slab decomposition -- */

/* One grid split along its slowest axis into n_slabs sub-domains (slabs),
 * each stepped by its own launches with halo rows exchanged between
 * neighbours after every launch: the decomposition a grid too large for one
 * GPU would take across several GPUs (one slab per GPU, the halo exchange a
 * peer copy), run here with every slab on the current device.  The paper
 * runs on one GPU and has no such decomposition; it extends the paper's
 * iteration batches (Sec. III-A): a batch graph of S iterations holds every
 * slab's kernel nodes and the halo copy nodes between them, so each slab's
 * next kernel waits only on its own previous kernel and the copies into and
 * out of its fields, and the slabs' kernels of one step can run at once.
 *
 * Split axis: y (rows) for GS_HEAT2D, z (planes) for GS_HEAT3D and GS_FDTD3D.
 * Slab s owns a contiguous range of rows/planes (sizes differing by at most
 * one, lower slabs the larger) and stores `halo` extra rows/planes on each
 * side it shares with a neighbour.  Thermal: halo = the largest temporal
 * depth the plans will use (a depth-t launch needs t halo rows, refreshed
 * from the neighbour after each launch); every slab must own >= halo rows.
 * FDTD: halo must be 1 (H's plane below a slab is refreshed after the H
 * update, E's plane above after the E update); with N cells the N+1 array
 * planes are partitioned, every slab owning >= 1.
 * Results are bit-identical to an undivided context of the same grid, plan
 * (depth, kernel) and coefficients, for every n_slabs, batch size, remainder
 * and PDL setting.
 * Memory: the slab set allocates and owns its fields (each slab's rows plus
 * halos; the FDTD components of a slab in one allocation); the caller moves
 * data with gs_slab_upload / gs_slab_read_field (dense host arrays of the
 * whole grid). */
typedef struct gs_slab gs_slab;

/* Create a slab set.  kind, sizes, storage, bc, stream: as gs_create
 * (stream NULL: the set creates its own); n_slabs in [1, 64]; halo as above.
 * The FDTD source is off until gs_slab_set_fdtd_params.  Errors:
 * GS_ERR_INVALID_ARG (sizes, a slab owning too few rows), GS_ERR_CUDA,
 * GS_ERR_OOM; message in gs_last_error(NULL); *out NULL on failure. */
gs_status gs_slab_create(gs_slab **out, gs_kind kind, int64_t nx, int64_t ny, int64_t nz, gs_dtype storage, gs_bc bc,
                         int32_t n_slabs, int32_t halo, void *stream);

/* Synchronise, free every slab's graphs, contexts and fields.  NULL is a no-op. */
gs_status gs_slab_destroy(gs_slab *s);

/* Message of the last failed call on s ("" if none). */
const char *gs_slab_last_error(const gs_slab *s);

/* The rows (2D) or planes (3D, FDTD arrays) slab k owns: [*first, *first + *count). */
gs_status gs_slab_extent(const gs_slab *s, int32_t k, int64_t *first, int64_t *count);

/* As gs_set_heat_coeffs / gs_set_fdtd_params (source cell in global
 * coordinates; the slab that owns its plane applies it) / gs_set_plan for
 * every slab.  gs_slab_set_plan: temporal_depth must not exceed the halo
 * (GS_ERR_UNSUPPORTED), and graph_loop and device_launch are not provided
 * for slab sets (GS_ERR_UNSUPPORTED); use_pdl applies to the per-step
 * launches, while a batch graph's kernel nodes follow copy nodes, whose
 * edges are full dependencies. */
gs_status gs_slab_set_heat_coeffs(gs_slab *s, const gs_heat_coeffs *c);
gs_status gs_slab_set_fdtd_params(gs_slab *s, const gs_fdtd_params *p);
gs_status gs_slab_set_plan(gs_slab *s, const gs_plan *plan);

/* Copy a dense float32 host array of the whole grid (as gs_upload for an
 * undivided context: T/T0/T1 or P, or an FDTD component) into every slab's
 * rows and halos.  GS_FIELD_T is the buffer holding the current state.
 * Synchronous. */
gs_status gs_slab_upload(gs_slab *s, gs_field id, const float *host, int64_t n);

/* Gather the rows every slab owns into a dense float32 host array of the
 * whole grid.  Synchronous. */
gs_status gs_slab_read_field(gs_slab *s, gs_field id, float *host_out, int64_t n);

/* Advance n_iters iterations: batch_size 0, per-step launches of every slab
 * followed by the halo copies; batch_size S > 0, floor(n/S) launches of a
 * cached batch graph and one remainder graph of n mod S iterations, as
 * gs_step.  Asynchronous. */
gs_status gs_slab_step(gs_slab *s, int64_t n_iters, int64_t batch_size);

/* FDTD time index of the next step (written to every slab's counter). */
gs_status gs_slab_set_time(gs_slab *s, int64_t n);

gs_status gs_slab_sync(gs_slab *s);

/* Counters of the set: graphs built and launched, kernel launches (per-step
 * path, summed over slabs), iterations; last_build_nodes counts the kernel
 * and copy nodes of the last batch graph. */
gs_status gs_slab_get_stats(const gs_slab *s, gs_stats *out);

/* -------------------------------------------- step without allocation -- */

/* The paper has no counterpart to this entry point: it serves callers that
 * cannot call cudaMalloc.  Code whose device memory all comes from its own
 * allocator or a fixed budget (a framework that forbids raw allocations
 * outside its memory manager), or a latency-critical loop that cannot afford
 * cudaMalloc's implicit device synchronisation, can still advance a batch of
 * 2D grids with the GS_MULTI_FUSED kernel here: the call allocates nothing.
 * Its descriptor table lives in a fixed array of GS_NOALLOC_MAX_INSTANCES
 * rows in device memory that belongs to the loaded library (every GPU that
 * loads the library holds it, about 14 KiB, until the process exits). */
#define GS_NOALLOC_MAX_INSTANCES 256

typedef struct gs_instance {
    void *T0;         /* ping-pong buffers, ny rows of `pitch` elements */
    void *T1;
    const void *P;    /* power map, ny rows of `p_pitch` elements */
    int64_t nx, ny;   /* grid size, each in [1, 2^20] */
    int64_t pitch;    /* elements per row of T0/T1 (>= nx, multiple of 16 bytes) */
    int64_t p_pitch;  /* elements per row of P (same rules) */
} gs_instance;

/* Advance n_inst independent 2D thermal grids by n_iters iterations, one
 * fused launch per iteration (block 64 threads, 8 rows per work item), on
 * `stream` (NULL: the legacy default stream).  parity: which buffer holds
 * the current state of every instance (0: T0); *parity_out (may be NULL)
 * receives the parity after the call.  Same update and results, bit for bit,
 * as gs_multi_step in GS_MULTI_FUSED mode.  Asynchronous.
 * Buffers: T0 and T1 occupy ny*pitch elements each and P ny*p_pitch; no
 * buffer may overlap another one, of the same instance or of another, except
 * that P buffers may overlap other P buffers (they are only read).
 * Set-up: the first call on a device (with a n_iters > 0) resolves the
 * table's device address (cudaGetSymbolAddress), the SM count and the step
 * kernel's occupancy with that device current, and loads the kernels; later
 * calls in the same CUDA context reuse them (a new context on the device,
 * e.g. after cudaDeviceReset, gets a new set-up on its first call).  Make
 * that first call on each device before any stream capture and before
 * relying on the call doing no set-up work.
 * Each call writes the table with at most four small fill launches whose
 * parameters carry the rows (nothing refers to the caller's memory after
 * the call returns), then launches one step per iteration.
 * Sharing: every call writes the same table (stream-ordered on its own
 * stream) and the table keeps the last call's contents; calls that overlap
 * on the GPU (different streams, or host threads racing) race on it.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Errors (message in gs_last_error(NULL)): GS_ERR_INVALID_ARG for n_inst
 * outside [1, GS_NOALLOC_MAX_INSTANCES], bad pointers, sizes or pitches,
 * overlapping buffers, or more than 2^31 work items; GS_ERR_NUMERIC for
 * non-finite coefficients; GS_ERR_CUDA if a CUDA call fails. */
gs_status gs_multi_step_noalloc(const gs_instance *inst, int32_t n_inst, int32_t parity, int64_t n_iters,
                                const gs_heat_coeffs *coeffs, gs_dtype storage, gs_bc bc, void *stream,
                                int32_t *parity_out);

/* --------------------------------------------------- fault injection -- */

/* Host-side fault injection for tests of the library's error paths (the
 * paper has no counterpart).  Every device allocation of the library
 * (contexts' scratch, instance-batch tables, slab fields, tuner snapshots,
 * cost-model buffers) and every kernel node it adds to a graph goes through
 * a wrapper; gs_debug_inject_failure(call, after) lets the next `after`
 * calls of that kind succeed and makes the one after them fail, once
 * (GS_INJECT_MALLOC: as cudaErrorMemoryAllocation; GS_INJECT_GRAPH_NODE: as
 * cudaErrorInvalidValue), with no CUDA call made for it; the injection is
 * then disarmed.  GS_INJECT_NONE disarms.  Process-wide; meant for a test
 * that owns the process's library calls while armed.  Nothing on the GPU
 * faults: the failure is a returned status.  gs_debug_injection_pending
 * tells whether an armed failure has not fired yet.  Errors:
 * GS_ERR_INVALID_ARG (unknown kind, after < 0, NULL). */
typedef enum gs_inject { GS_INJECT_NONE = 0, GS_INJECT_MALLOC = 1, GS_INJECT_GRAPH_NODE = 2 } gs_inject;
gs_status gs_debug_inject_failure(gs_inject call, int64_t after);
gs_status gs_debug_injection_pending(int32_t *pending);

/* Bounds-checked builds (libgraphstep_checked.so, compiled with GS_CHECKED
 * by `python paper_2501_09398_gb300/build.py --checked`; the paper has no
 * counterpart): every global field access of the thermal and FDTD stencil
 * kernels (loads, stores, material ids; not the STREAM kernel's tensor
 * copies, which the tensor map itself keeps inside the field: reads outside
 * its nx x ny x nz elements are filled with zeros) is checked against a table of up to
 * GS_CHECK_MAX_RANGES byte ranges [lo, hi) of device memory the caller
 * registers: its field buffers and the device memory a context owns
 * (gs_debug_owned_ranges: the FDTD fused plan's second set, once a step has
 * set it up).  An access outside every range is counted, its address
 * recorded and the access skipped (a load gives zeros), so nothing faults.
 * gs_debug_check_ranges replaces the table and clears the count;
 * gs_debug_check_read returns the count of refused accesses since, and the
 * first refused address, and clears the count.  gs_debug_checked_build
 * returns 1 in a checked build, 0 otherwise; in an ordinary build the two
 * calls return GS_ERR_UNSUPPORTED.  Errors: GS_ERR_INVALID_ARG (NULL, n
 * outside [0, GS_CHECK_MAX_RANGES], lo > hi), GS_ERR_CUDA. */
#define GS_CHECK_MAX_RANGES 128
int gs_debug_checked_build(void);
/* The byte ranges of device memory ctx owns that its kernels read or write
 * (the fused FDTD plan's second set of components); *n_out gets their
 * number, up to `capacity` are written.  Any build. */
gs_status gs_debug_owned_ranges(const gs_ctx *ctx, uint64_t *lo, uint64_t *hi, int32_t capacity, int32_t *n_out);
gs_status gs_debug_check_ranges(const uint64_t *lo, const uint64_t *hi, int32_t n);
gs_status gs_debug_check_read(uint64_t *refused, uint64_t *first_refused_address);

/* Bounded waits inside the library's kernels (the STREAM kernel's waits for
 * its tensor copies, the paper has no counterpart): a wait gives up after
 * about one second of the GPU's global timer instead of hanging; its block
 * then stops early, so the launch's results are not defined.  *count_out
 * gets the number of blocks whose wait ran out since the previous call, and
 * the count is cleared.  Synchronises the device.  Errors:
 * GS_ERR_INVALID_ARG (NULL), GS_ERR_CUDA. */
gs_status gs_wait_timeouts(uint64_t *count_out);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHSTEP_H */
