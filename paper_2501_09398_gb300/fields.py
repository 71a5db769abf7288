"""Caller-owned device memory for a context's fields, allocated with PyTorch.

The library borrows these buffers (gs_bind_field); the objects below only
allocate pitched tensors of the right size and bind them.  Keep the object
alive while the context uses the fields.
"""
from __future__ import annotations

import torch

from . import (GS_BF16, GS_F16, GS_F32, GS_FIELD_MAT, GS_FIELD_P, GS_FIELD_T0, GS_FIELD_T1, FDTD_FIELDS,
               gs_bind_field, gs_multi_bind_field, gs_required_pitch)

_TORCH = {GS_F32: torch.float32, GS_BF16: torch.bfloat16, GS_F16: torch.float16}


def _alloc(rows: int, pitch: int, dtype: int, device) -> torch.Tensor:
    # torch allocations are at least 256-byte aligned, so rows start on 16 bytes
    return torch.zeros(rows * pitch, dtype=_TORCH[dtype], device=device)


def _ready(device) -> None:
    # The zero fill runs on PyTorch's stream; a context with its own
    # non-blocking stream must not see the buffers before it finishes.
    torch.cuda.current_stream(torch.device(device)).synchronize()


class HeatFields:
    """T0, T1 (nz*ny rows) and P (ny rows), all with the same pitch."""

    def __init__(self, ctx, nx: int, ny: int, nz: int = 1, dtype: int = GS_F32, device="cuda", pitch: int = 0):
        self.pitch = pitch or gs_required_pitch(dtype, nx)
        self.nx, self.ny, self.nz, self.dtype = nx, ny, nz, dtype
        self.T0 = _alloc(ny * nz, self.pitch, dtype, device)
        self.T1 = _alloc(ny * nz, self.pitch, dtype, device)
        self.P = _alloc(ny, self.pitch, dtype, device)
        gs_bind_field(ctx, GS_FIELD_T0, self.T0.data_ptr(), self.pitch)
        gs_bind_field(ctx, GS_FIELD_T1, self.T1.data_ptr(), self.pitch)
        gs_bind_field(ctx, GS_FIELD_P, self.P.data_ptr(), self.pitch)
        _ready(device)

    def bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.T0, self.T1, self.P))


class FdtdFields:
    """Six (N+1)^3 Yee components with a common pitch and, with media=True,
    the uint8 material map (same pitch in elements)."""

    def __init__(self, ctx, N: int, dtype: int = GS_F32, device="cuda", pitch: int = 0, media: bool = False):
        self.pitch = pitch or gs_required_pitch(dtype, N + 1)
        self.N, self.dtype = N, dtype
        self.f = [_alloc((N + 1) * (N + 1), self.pitch, dtype, device) for _ in range(6)]
        for fid, t in zip(FDTD_FIELDS, self.f):
            gs_bind_field(ctx, fid, t.data_ptr(), self.pitch)
        self.mat = None
        if media:
            self.mat = torch.zeros((N + 1) * (N + 1) * self.pitch, dtype=torch.uint8, device=device)
            gs_bind_field(ctx, GS_FIELD_MAT, self.mat.data_ptr(), self.pitch)
        _ready(device)

    def bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.f + ([self.mat] if self.mat is not None else []))


class MultiFields:
    """T0, T1, P of every instance of a gs_multi batch (2D, square or not)."""

    def __init__(self, m, nx, ny, dtype: int = GS_F32, device="cuda"):
        self.bufs = []
        for i, (w, h) in enumerate(zip(nx, ny)):
            pitch = gs_required_pitch(dtype, w)
            t0, t1, p = (_alloc(h, pitch, dtype, device) for _ in range(3))
            gs_multi_bind_field(m, i, GS_FIELD_T0, t0.data_ptr(), pitch)
            gs_multi_bind_field(m, i, GS_FIELD_T1, t1.data_ptr(), pitch)
            gs_multi_bind_field(m, i, GS_FIELD_P, p.data_ptr(), pitch)
            self.bufs.append((t0, t1, p))
        _ready(device)
