"""Small parity cases of every stencil kernel variant, run once with the
ordinary library and once with the bounds-checked build (GS_LIBRARY=checked,
in a process of its own): each returns its output field(s) and, in the
checked build, the count of refused accesses.  Shared by
test_checked_gpu.py and checked_run.py."""
import numpy as np

import gs_inputs


def _span(t):
    return (t.data_ptr(), t.data_ptr() + t.numel() * t.element_size())


def _stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


def heat(g, nx, ny, nz, n, S, plan, dtype="f32", bc=0, omit_p=False):
    kind = g.GS_HEAT2D if nz == 1 else g.GS_HEAT3D
    ctx = g.gs_create(kind, nx, ny, nz, g.DTYPES[dtype], bc, _stream())
    f = g.HeatFields(ctx, nx, ny, nz, g.DTYPES[dtype])
    try:
        g.gs_set_plan(ctx, **plan)
        T, P = gs_inputs.heat_fields(nx, ny, nz, seed=nx + ny + nz)
        g.gs_upload(ctx, g.GS_FIELD_T, T)
        g.gs_upload(ctx, g.GS_FIELD_P, P)
        checked = g.gs_debug_checked_build()
        if checked:
            g.gs_debug_check_ranges([_span(f.T0), _span(f.T1)] + ([] if omit_p else [_span(f.P)]))
        g.gs_step(ctx, n, S)
        out = g.gs_read_field(ctx, g.GS_FIELD_T, np.empty_like(T))
        refused = g.gs_debug_check_read() if checked else (0, 0)
        return [out], refused, _span(f.P)
    finally:
        g.gs_destroy(ctx)
        del f


def fdtd(g, N, n, S, plan, dtype="f32", media=False):
    ctx = g.gs_create(g.GS_FDTD3D, N, N, N, g.DTYPES[dtype], g.GS_BC_PEC, _stream())
    f = g.FdtdFields(ctx, N, g.DTYPES[dtype], media=media)
    try:
        g.gs_set_fdtd_params(ctx, courant=0.5, src_on=1, src=(N // 2, N // 3, N - 1))
        if media:
            mat, table = gs_inputs.fdtd_media(N, n_mat=3, n_boxes=5, seed=2)
            g.gs_set_fdtd_media(ctx, table)
            g.gs_upload_u8(ctx, g.GS_FIELD_MAT, mat)
        g.gs_set_plan(ctx, **plan)
        init = gs_inputs.fdtd_random_all(N, seed=N)
        for fid, name in zip(g.FDTD_FIELDS, ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")):
            g.gs_upload(ctx, fid, np.ascontiguousarray(init[name], dtype=np.float32))
        g.gs_step(ctx, 0, 0)  # sets up the launches (and a fused plan's second set)
        checked = g.gs_debug_checked_build()
        if checked:
            spans = [_span(t) for t in f.f] + ([_span(f.mat)] if media else []) + g.gs_debug_owned_ranges(ctx)
            g.gs_debug_check_ranges(spans)
        g.gs_step(ctx, n, S)
        outs = [g.gs_read_field(ctx, fid, np.empty((N + 1,) * 3, dtype=np.float32)) for fid in g.FDTD_FIELDS]
        refused = g.gs_debug_check_read() if checked else (0, 0)
        return outs, refused, None
    finally:
        g.gs_destroy(ctx)
        del f


def multi(g, dims, n, S, plan):
    import torch

    nx, ny = [d[0] for d in dims], [d[1] for d in dims]
    m = g.gs_multi_create(nx, ny, g.GS_F32, g.GS_BC_CLAMP, torch.cuda.current_stream().cuda_stream)
    bufs = g.MultiFields(m, nx, ny)
    try:
        g.gs_multi_set_plan(m, **plan)
        fields = [gs_inputs.heat_fields(w, h, 1, seed=60 + i) for i, (w, h) in enumerate(dims)]
        for i, (T, P) in enumerate(fields):
            g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
        checked = g.gs_debug_checked_build()
        if checked:
            g.gs_debug_check_ranges([_span(t) for trio in bufs.bufs for t in trio])
        g.gs_multi_step(m, n, S, g.GS_MULTI_FUSED)
        outs = [g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in enumerate(fields)]
        refused = g.gs_debug_check_read() if checked else (0, 0)
        return outs, refused, None
    finally:
        g.gs_multi_destroy(m)
        del bufs


K_MARCH, K_WAVE, K_TILE, K_COLUMN, K_SMEM, K_FUSED, K_STREAM = 1, 2, 3, 4, 5, 6, 7


def cases():
    """(name, function of the package) for every case."""
    out = []
    for bc in (0, 1):
        for nx, ny, nz in ((77, 45, 1), (40, 33, 5), (29, 13, 8), (33, 20, 19)):
            deep = nz > 8
            plans = [dict(kernel=K_COLUMN, rows=1), dict(kernel=K_COLUMN, rows=8), dict(kernel=K_MARCH, block_x=32, rows=5),
                     dict(kernel=K_TILE, temporal_depth=2, tile_x=13, tile_y=7),
                     dict(kernel=K_TILE, temporal_depth=4, tile_x=16, tile_y=8)]
            if not deep:
                plans += [dict(kernel=K_SMEM, rows=3), dict(kernel=K_WAVE, rows=3, block_x=64),
                          dict(kernel=K_WAVE, temporal_depth=2, rows=3, block_x=64),
                          dict(kernel=K_WAVE, temporal_depth=4, rows=16, block_x=32),
                          dict(kernel=K_COLUMN, temporal_depth=2, block_x=64, rows=2),
                          dict(kernel=K_COLUMN, temporal_depth=2, block_x=256),
                          dict(kernel=K_COLUMN, temporal_depth=4, block_x=32)]
            else:
                plans += [dict(kernel=K_COLUMN, temporal_depth=2, block_x=128, tile_y=5),
                          dict(kernel=K_COLUMN, temporal_depth=2, block_x=32, tile_y=32)]
            if nz > 1:  # planes streamed through shared memory (any stack depth)
                plans += [dict(kernel=K_STREAM, temporal_depth=2, block_x=256, tile_y=3),
                          dict(kernel=K_STREAM, temporal_depth=2, block_x=512, tile_y=32)]
            for i, p in enumerate(plans):
                out.append((f"heat {nx}x{ny}x{nz} bc{bc} plan{i}",
                            lambda g, a=(nx, ny, nz), p=p, bc=bc: heat(g, *a, 11, 4, p, bc=bc)))
    for nx, ny, nz in ((130, 20, 1), (40, 33, 8)):
        out.append((f"heat {nx}x{ny}x{nz} bf16 column2",
                    lambda g, a=(nx, ny, nz): heat(g, *a, 9, 4, dict(kernel=K_COLUMN, temporal_depth=2), dtype="bf16")))
    out.append(("heat 200x30x12 bf16 stream2",
                lambda g: heat(g, 200, 30, 12, 9, 4, dict(kernel=K_STREAM, temporal_depth=2, block_x=256, tile_y=5),
                               dtype="bf16")))
    for N in (37, 128):
        for i, p in enumerate((dict(kernel=K_COLUMN, rows=1), dict(kernel=K_COLUMN, rows=8),
                               dict(kernel=K_MARCH, rows=4, block_x=32), dict(kernel=K_FUSED, rows=2),
                               dict(kernel=K_FUSED, rows=4, tile_y=6))):
            out.append((f"fdtd {N} plan{i}", lambda g, N=N, p=p: fdtd(g, N, 5, 2, p)))
    out.append(("fdtd 20 media", lambda g: fdtd(g, 20, 5, 2, dict(kernel=K_COLUMN, rows=2), media=True)))
    out.append(("fdtd 20 media fused march",
                lambda g: fdtd(g, 20, 5, 2, dict(kernel=K_FUSED, rows=2, tile_y=4), media=True)))
    out.append(("fdtd 16 f16 fused", lambda g: fdtd(g, 16, 7, 3, dict(kernel=K_FUSED), dtype="f16")))
    out.append(("fdtd 16 bf16 fused march", lambda g: fdtd(g, 16, 7, 3, dict(kernel=K_FUSED, tile_y=3), dtype="bf16")))
    dims = [(130, 17), (5, 9), (64, 64)]
    for i, p in enumerate((dict(kernel=K_MARCH), dict(kernel=K_COLUMN, rows=4),
                           dict(kernel=K_COLUMN, rows=2, temporal_depth=2))):
        out.append((f"multi plan{i}", lambda g, p=p: multi(g, dims, 9, 4, p)))
    return out
