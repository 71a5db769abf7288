"""CPU re-trace of the data flow of the temporally blocked thermal kernels
(a launch advances t time levels): the COLUMN kernel at depth 2 and 4 (2D),
the WAVE kernel at depths 1, 2 and 4 (2D and 3D) and the TILE kernel
(2D and 3D).

Each test follows one launch's blocks level by level and marks which values
are the true level-s values of their cells.  A level-0 value is valid when
its cell lies in the grid and was loaded from its own address (not from a
clamped one).  A level-s value is valid when its cell lies in the grid, the
kernel computes that row at level s, and every operand it reads is valid at
level s-1 or is the boundary value the kernel substitutes at the grid's
edge.  The operands are the cell itself, the x-neighbours (registers, or a
shuffle from the next lane, which at a warp edge returns the lane's own
value and so is never valid), the y-neighbours (the kernel's row registers
or march window), the z-neighbours (3D) and the P value of the row.  Every
cell a launch stores must be valid at level t.  The formulas restate the
kernels' tiles, halos and level schedules (csrc/heat.cu); a change to
either is checked here before it runs on a GPU."""
import numpy as np
import pytest

VEC = {4: 4, 2: 8}  # elements per 16-byte vector by element size


def _x_neighbours(prev, x, nx):
    """West and east operands' validity for (..., lane, row, element)
    arrays: the element beside, or the next lane's edge element by shuffle
    (lanes 0 and 31 have no lane beyond them), or the boundary value at
    x = 0 and x = nx - 1."""
    west = np.zeros_like(prev)
    east = np.zeros_like(prev)
    west[..., 1:] = prev[..., :-1]
    west[..., 1:, :, 0] = prev[..., :-1, :, -1]
    east[..., :-1] = prev[..., 1:]
    east[..., :-1, :, -1] = prev[..., 1:, :, 0]
    return west | (x == 0), east | (x + 1 >= nx)


def _y_neighbours(prev, y, ny):
    north = np.zeros_like(prev)
    south = np.zeros_like(prev)
    north[..., 1:, :] = prev[..., :-1, :]
    south[..., :-1, :] = prev[..., 1:, :]
    return north | (y == 0), south | (y + 1 >= ny)


# ------------------------------------------------ COLUMN, depth T (2D) ----

def column_t_block_valid(nx, ny, V, T, R, BY, bx, by):
    """Level-T validity and store mask of every warp row of block (bx, by):
    arrays (BY, 32, NR, V) over warp row, lane, row register, element."""
    NR = R + 2 * T
    xs = bx * 30 * V - V
    lane = np.arange(32)[None, :, None, None]
    x0 = xs + lane * V
    x = x0 + np.arange(V)[None, None, None, :]
    y0 = ((by * BY + np.arange(BY)) * R)[:, None, None, None]
    k = np.arange(NR)[None, None, :, None]
    y = y0 - T + k
    ing = (x >= 0) & (x < nx) & (y >= 0) & (y < ny)
    # loads at clamped coordinates: the lane's own vector when x0 >= 0
    # (x0 < nx for a lane with a cell in the grid); rows clamped into the
    # grid are only the true rows when y is in the grid
    valid = ing & (x0 >= 0)
    pvalid = valid & (k >= 1) & (k <= NR - 2)  # P rows 1 .. NR-2 are loaded
    for s in range(1, T + 1):
        north, south = _y_neighbours(valid, y, ny)
        west, east = _x_neighbours(valid, x, nx)
        updated = (k >= s) & (k <= NR - 1 - s)  # rows the level updates in place
        valid = updated & ing & valid & north & south & west & east & pvalid
    stored = (lane >= 1) & (lane <= 30) & (x0 < nx) & (k >= T) & (k < T + R) & (y < ny) & (x < nx)
    return valid, np.broadcast_to(stored, valid.shape), x, y


@pytest.mark.parametrize("nx,ny", [(300, 37), (96, 64), (77, 45), (500, 130), (3, 2), (1, 9), (130, 17),
                                   (241, 8), (121, 5)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("depth", [2, 4])
@pytest.mark.parametrize("block_x", [32, 64, 256])
def test_column_t_stores_only_valid_cells(nx, ny, esize, depth, block_x):
    V = VEC[esize]
    R = 4 if V == 4 else 2
    BY = max(1, min(block_x // 32, 8))
    covered = np.zeros((ny, nx), dtype=np.int64)
    for bx in range(-(-nx // (30 * V))):
        for by in range(-(-ny // (R * BY))):
            valid, stored, x, y = column_t_block_valid(nx, ny, V, depth, R, BY, bx, by)
            assert np.all(valid[stored]), (bx, by)
            xb = np.broadcast_to(x, stored.shape)[stored]
            yb = np.broadcast_to(y, stored.shape)[stored]
            np.add.at(covered, (yb, xb), 1)
    assert np.all(covered == 1)


# ------------------------------------------------------ WAVE, depth T ----

def wave_block_valid(nx, ny, nz, V, T, R, WB, bx, by):
    """Level-T validity and store mask of block (bx, by) of the wavefront
    kernel: arrays (planes or warp rows, 32, rows, V) over the global rows
    q in [y0 - 2T, y0 + R + T) of each warp."""
    is3d = nz > 1
    W = nz if is3d else WB
    xs = bx * 30 * V - V
    lane = np.arange(32)[None, :, None, None]
    x0 = xs + lane * V
    x = x0 + np.arange(V)[None, None, None, :]
    w = np.arange(W)[:, None, None, None]
    y0 = by * R + 0 * w if is3d else (by * WB + w) * R
    rbeg = y0 - T  # first level-0 row of the march
    nsteps = R + 2 * T
    q = y0 - 2 * T + np.arange(R + 3 * T)[None, None, :, None]  # rows any level touches
    ld_ok = (x0 >= 0) & (x0 < nx)
    ing = (x >= 0) & (x < nx) & (q >= 0) & (q < ny)
    marched = (q >= rbeg) & (q < rbeg + nsteps)  # level-0 rows (and P rows) loaded
    valid = ing & ld_ok & marched
    has_p = (w == 0) if is3d else np.ones_like(w, dtype=bool)
    pvalid = (ing & ld_ok & marched) | (~has_p)  # 3D planes above 0 add no P
    for s in range(1, T + 1):
        north, south = _y_neighbours(valid, q, ny)
        west, east = _x_neighbours(valid, x, nx)
        down = np.ones_like(valid)
        up = np.ones_like(valid)
        if is3d:  # planes z - 1 and z + 1 of the same row and level, or the boundary value
            down[1:] = valid[:-1]
            up[:-1] = valid[1:]
        computed = (q >= rbeg - s) & (q <= rbeg + nsteps - 1 - s)  # rows level s computes
        valid = computed & ing & valid & north & south & west & east & down & up & pvalid
    stored = (lane >= 1) & (lane <= 30) & (x0 < nx) & (q >= y0) & (q < y0 + R) & (q < ny) & (x < nx)
    return valid, np.broadcast_to(stored, valid.shape), x, q, w


@pytest.mark.parametrize("nx,ny,nz", [(300, 37, 1), (77, 45, 1), (3, 2, 1), (130, 17, 1), (500, 9, 1),
                                      (131, 19, 3), (64, 10, 8), (250, 7, 16), (5, 5, 2), (121, 4, 1)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("depth", [1, 2, 4])
@pytest.mark.parametrize("block_x,rows", [(64, 4), (128, 32), (32, 1), (96, 7)])
def test_wave_stores_only_valid_cells(nx, ny, nz, esize, depth, block_x, rows):
    V = VEC[esize]
    is3d = nz > 1
    WB = nz if is3d else max(1, block_x // 32)
    ry = rows if is3d else rows * WB
    covered = np.zeros((nz, ny, nx), dtype=np.int64)
    for bx in range(-(-nx // (30 * V))):
        for by in range(-(-ny // ry)):
            valid, stored, x, q, w = wave_block_valid(nx, ny, nz, V, depth, rows, WB, bx, by)
            assert np.all(valid[stored]), (bx, by)
            z = np.broadcast_to(w if is3d else 0 * w, stored.shape)[stored]
            np.add.at(covered, (z, np.broadcast_to(q, stored.shape)[stored],
                                np.broadcast_to(x, stored.shape)[stored]), 1)
    assert np.all(covered == 1)


# ---------------------------------------------------- TILE, depth D ----

@pytest.mark.parametrize("nx,ny,nz", [(37, 23, 1), (64, 64, 1), (5, 3, 1), (30, 17, 4), (9, 11, 20)])
@pytest.mark.parametrize("depth", [2, 4])
@pytest.mark.parametrize("tile", [(16, 8), (32, 32), (7, 5)])
def test_tile_stores_only_valid_cells(nx, ny, nz, depth, tile):
    # heat_temporal_kernel: a block loads its tile plus a D-wide halo
    # (cells outside the grid left invalid), updates the shrinking window
    # [s, I - s) at level s (skipping cells outside the grid), and stores
    # the tile interior
    tx, ty = tile
    IX, IY = tx + 2 * depth, ty + 2 * depth
    covered = np.zeros((nz, ny, nx), dtype=np.int64)
    for bx in range(-(-nx // tx)):
        for by in range(-(-ny // ty)):
            gx = (bx * tx - depth + np.arange(IX))[None, None, :]
            gy = (by * ty - depth + np.arange(IY))[None, :, None]
            iz = np.arange(nz)[:, None, None]
            ix = np.arange(IX)[None, None, :]
            iy = np.arange(IY)[None, :, None]
            ing = (gx >= 0) & (gx < nx) & (gy >= 0) & (gy < ny) & (iz >= 0)
            valid = ing.copy()
            pvalid = ing | (iz > 0)  # the P tile feeds plane 0 only
            for s in range(1, depth + 1):
                west = np.zeros_like(valid)
                east = np.zeros_like(valid)
                west[..., 1:] = valid[..., :-1]
                east[..., :-1] = valid[..., 1:]
                north, south = _y_neighbours(valid, gy, ny)
                down = np.ones_like(valid)
                up = np.ones_like(valid)
                down[1:] = valid[:-1]
                up[:-1] = valid[1:]
                window = (ix >= s) & (ix < IX - s) & (iy >= s) & (iy < IY - s)
                valid = (window & ing & valid & (west | (gx == 0)) & (east | (gx + 1 >= nx)) & north & south
                         & down & up & pvalid)
            stored = (ix >= depth) & (ix < depth + tx) & (iy >= depth) & (iy < depth + ty) & (gx < nx) & (gy < ny)
            stored = np.broadcast_to(stored, valid.shape)
            assert np.all(valid[stored]), (bx, by)
            np.add.at(covered, (np.broadcast_to(iz, stored.shape)[stored], np.broadcast_to(gy, stored.shape)[stored],
                                np.broadcast_to(gx, stored.shape)[stored]), 1)
    assert np.all(covered == 1)


@pytest.mark.parametrize("esize", [4, 2])
def test_halo_lanes_bound_the_depth(esize):
    # the kernels' static_assert(T <= V): lanes 0 and 31 lose one cell of
    # validity per level at each warp edge, so at depth V + 1 the loss
    # reaches the stored lanes 1 and 30
    V = VEC[esize]
    nx, ny = 40 * 30 * V, 40  # interior blocks, away from every x edge
    for T, ok in ((V, True), (V + 1, False)):
        valid, stored, _, _, _ = wave_block_valid(nx, ny, 1, V, T, 4, 1, 1, 1)
        assert bool(np.all(valid[stored])) == ok, ("wave", T)
        valid, stored, _, _ = column_t_block_valid(nx, ny, V, T, 2, 1, 1, 1)
        assert bool(np.all(valid[stored])) == ok, ("column", T)
