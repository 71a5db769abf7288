"""Helpers for the GPU tests: run the library through its C ABI on seeded
inputs and compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np

# Tolerances.  Thermal FP32: max relative error <= 1e-5 after 1000 steps;
# FDTD FP32: relative L2 error <= 1e-4 after 5000 steps (all six
# components concatenated).
HEAT_RTOL = 1e-5
FDTD_RL2 = 1e-4


def gs():
    import paper_2501_09398_gb300 as g

    return g


def stream_handle():
    import torch

    return torch.cuda.current_stream().cuda_stream


def heat_setup(nx, ny, nz=1, dtype="f32", bc=0, kind=None, plan=None, coeffs=None):
    g = gs()
    if kind is None:
        kind = g.GS_HEAT2D if nz == 1 else g.GS_HEAT3D
    ctx = g.gs_create(kind, nx, ny, nz, g.DTYPES[dtype], bc, stream_handle())
    fields = g.HeatFields(ctx, nx, ny, nz, g.DTYPES[dtype])
    if coeffs is not None:
        g.gs_set_heat_coeffs(ctx, **coeffs)
    if plan:
        g.gs_set_plan(ctx, **plan)
    return ctx, fields


def heat_upload(ctx, T0, P):
    g = gs()
    g.gs_upload(ctx, g.GS_FIELD_T, np.ascontiguousarray(T0, dtype=np.float32))
    g.gs_upload(ctx, g.GS_FIELD_P, np.ascontiguousarray(P, dtype=np.float32))


def heat_read(ctx, shape):
    g = gs()
    out = np.empty(shape, dtype=np.float32)
    return g.gs_read_field(ctx, g.GS_FIELD_T, out)


def heat_gpu(T0, P, n, S=0, dtype="f32", bc=0, plan=None, coeffs=None, kind=None):
    """Run n steps on the GPU from (T0, P); return the float32 result."""
    g = gs()
    nz = 1 if T0.ndim == 2 else T0.shape[0]
    ny, nx = T0.shape[-2:]
    ctx, fields = heat_setup(nx, ny, nz, dtype, bc, kind, plan, coeffs)
    try:
        heat_upload(ctx, T0, P)
        g.gs_step(ctx, n, S)
        return heat_read(ctx, T0.shape)
    finally:
        g.gs_destroy(ctx)
        del fields


def max_rel(a, ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - ref) / np.abs(ref)))


def rel_l2(a, ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((np.asarray(a, dtype=np.float64) - ref).ravel()) / np.linalg.norm(ref.ravel()))


FDTD_NAMES = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def fdtd_setup(N, dtype="f32", plan=None, src=None, courant=0.5, media=None):
    """media: None, or (mat, table) as gs_inputs.fdtd_media returns."""
    g = gs()
    ctx = g.gs_create(g.GS_FDTD3D, N, N, N, g.DTYPES[dtype], g.GS_BC_PEC, stream_handle())
    fields = g.FdtdFields(ctx, N, g.DTYPES[dtype], media=media is not None)
    if media is not None:
        g.gs_set_fdtd_media(ctx, media[1])
        g.gs_upload_u8(ctx, g.GS_FIELD_MAT, media[0])
    if src is not None:
        g.gs_set_fdtd_params(ctx, courant=courant, src_on=1, src=src)
    else:
        g.gs_set_fdtd_params(ctx, courant=courant, src_on=0, src=(N // 2, N // 2, N // 2))
    if plan:
        g.gs_set_plan(ctx, **plan)
    return ctx, fields


def fdtd_upload(ctx, N, fields_np):
    g = gs()
    for fid, name in zip(g.FDTD_FIELDS, FDTD_NAMES):
        a = fields_np.get(name)
        if a is None:
            a = np.zeros((N + 1,) * 3, dtype=np.float32)
        g.gs_upload(ctx, fid, np.ascontiguousarray(a, dtype=np.float32))


def fdtd_read(ctx, N):
    g = gs()
    out = {}
    for fid, name in zip(g.FDTD_FIELDS, FDTD_NAMES):
        out[name] = g.gs_read_field(ctx, fid, np.empty((N + 1,) * 3, dtype=np.float32))
    return out


def fdtd_concat(f):
    return np.concatenate([np.asarray(f[n], dtype=np.float64).ravel() for n in FDTD_NAMES])
