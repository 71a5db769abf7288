"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the stepping arithmetic: it only draws random
numbers (numpy PCG64 via ``default_rng``) and rounds them to float32, so the
CUDA path and the FP64 oracle start from the same values.

The paper's Hotspot inputs (Rodinia temperature and power maps, Sec. III-C)
are not available; these distributions stand in for them:

* thermal field T ~ U[320, 340] (kelvin), power map P ~ U[0, 1e-3];
* uneven instance batches: square grids with side round(exp(U[ln 64, ln 1024])),
  instance k seeded with 1000 + k;
* FDTD: zero fields (the soft source drives the cavity) or, for the
  source-free pins, a random interior E field;
* FDTD media (the cavity filled with objects): material 0 is vacuum, the
  other materials are axis-aligned boxes placed at random (later boxes
  overwrite earlier ones) with eps_r ~ U[1.5, 8], mu_r ~ U[1, 2], and, for
  lossy materials, sigma ~ U[0, 0.05] and sigma_m ~ U[0, 0.02].
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 0
T_RANGE = (320.0, 340.0)
P_RANGE = (0.0, 1e-3)


def heat_fields(nx: int, ny: int, nz: int = 1, seed: int = DEFAULT_SEED):
    """Return (T, P) as float32 arrays: T (ny, nx) or (nz, ny, nx); P (ny, nx)."""
    rng = np.random.default_rng(seed)
    shape = (ny, nx) if nz == 1 else (nz, ny, nx)
    T = rng.uniform(*T_RANGE, size=shape).astype(np.float32)
    P = rng.uniform(*P_RANGE, size=(ny, nx)).astype(np.float32)
    return T, P


def instance_sides(n: int = 64, lo: int = 64, hi: int = 1024, seed: int = DEFAULT_SEED):
    """Side lengths of ``n`` square grids, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=n)
    return [int(min(hi, max(lo, round(math.exp(v))))) for v in u]


def instance_fields(sides, seed_base: int = 1000):
    """(T, P) float32 pairs for square instances; instance k uses seed seed_base + k."""
    return [heat_fields(s, s, 1, seed_base + k) for k, s in enumerate(sides)]


def fdtd_random_e(N: int, seed: int = DEFAULT_SEED):
    """Random interior E components (float32, (N+1)^3 each, [k][j][i]).

    Tangential E on the PEC walls is zero; entries outside each component's
    index range are zero.  Ex lives on i < N, 0 < j < N, 0 < k < N; Ey and Ez
    likewise with the roles of the axes rotated.
    """
    rng = np.random.default_rng(seed)
    m = N + 1
    out = {}
    for name, axis in (("Ex", 2), ("Ey", 1), ("Ez", 0)):
        a = rng.standard_normal((m, m, m)).astype(np.float32)
        mask = np.zeros((m, m, m), dtype=bool)
        # interior in the two transverse axes, [0, N) along the own axis
        sl = [slice(1, N), slice(1, N), slice(1, N)]
        sl[axis] = slice(0, N)
        mask[tuple(sl)] = True
        a[~mask] = 0.0
        out[name] = a
    return out


def fdtd_random_all(N: int, seed: int = DEFAULT_SEED):
    """Random values in every entry of all six components (float32,
    (N+1)^3 each, [k][j][i]), the PEC walls and the unused entries included.

    Not a physical state: a stress input for the arithmetic at the walls
    (entries the update never writes keep their values, and H next to a wall
    then sees non-zero tangential E)."""
    rng = np.random.default_rng(seed)
    m = N + 1
    return {name: rng.standard_normal((m, m, m)).astype(np.float32) for name in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")}


def fdtd_media(N: int, n_mat: int = 4, n_boxes: int = 8, lossy: bool = True, seed: int = DEFAULT_SEED,
               swap_symmetric: bool = False):
    """A material map (uint8, (N+1)^3, [k][j][i]) and its table of
    (eps_r, sigma, mu_r, sigma_m) rows; row 0 is vacuum.

    ``swap_symmetric`` mirrors every box across the plane i = j, so that the
    map is unchanged when i and j are swapped."""
    rng = np.random.default_rng(seed)
    table = [(1.0, 0.0, 1.0, 0.0)]
    for _ in range(1, n_mat):
        eps_r = float(np.float32(rng.uniform(1.5, 8.0)))
        mu_r = float(np.float32(rng.uniform(1.0, 2.0)))
        sigma = float(np.float32(rng.uniform(0.0, 0.05))) if lossy else 0.0
        sigma_m = float(np.float32(rng.uniform(0.0, 0.02))) if lossy else 0.0
        table.append((eps_r, sigma, mu_r, sigma_m))
    m = N + 1
    mat = np.zeros((m, m, m), dtype=np.uint8)
    for _ in range(n_boxes):
        lo = rng.integers(0, m, size=3)
        ext = rng.integers(1, max(2, m // 2), size=3)
        hi = np.minimum(lo + ext, m)
        mid = int(rng.integers(1, n_mat)) if n_mat > 1 else 0
        mat[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = mid
        if swap_symmetric:
            mat[lo[2]:hi[2], lo[0]:hi[0], lo[1]:hi[1]] = mid
    return mat, table


def round_to(arr: np.ndarray, dtype: str) -> np.ndarray:
    """Round float32 values to a storage dtype ('f32', 'bf16', 'f16') and back
    to float32 (round-to-nearest-even), via torch's CPU casts."""
    if dtype == "f32":
        return np.asarray(arr, dtype=np.float32)
    import torch

    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).to(tdt).float().numpy()
