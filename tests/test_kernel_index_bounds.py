"""CPU re-trace of the index arithmetic of the COLUMN kernels (thermal depth
1 in 2D, thin and chunked deep stacks; thermal depth 2 and 4 in 2D; the
FDTD H and E kernels in the aligned and general layouts): for every thread
of every block of the launch the library makes, every global load and store
must lie inside its buffer and inside its row (the pitch), and the stores of
a launch must cover every cell of the field exactly once.  The formulas
restate the kernels' address computations (csrc/heat.cu, csrc/fdtd.cu) for
ragged shapes, so that a change to either is checked here before it runs on
a GPU."""
import numpy as np
import pytest

VEC = {4: 4, 2: 8}  # elements per 16-byte vector by element size


def pitch_of(width, esize):
    per = 16 // esize
    return -(-width // per) * per


def threads(grid, block):
    """Arrays of (bx, by, bz, tx, ty, tz) for every thread of a launch."""
    g = np.stack(np.meshgrid(*[np.arange(n) for n in grid], indexing="ij"), -1).reshape(-1, 3)
    t = np.stack(np.meshgrid(*[np.arange(n) for n in block], indexing="ij"), -1).reshape(-1, 3)
    gi = np.repeat(g, len(t), axis=0)
    ti = np.tile(t, (len(g), 1))
    return gi[:, 0], gi[:, 1], gi[:, 2], ti[:, 0], ti[:, 1], ti[:, 2]


def warp_all(pred, bx, by, bz, ty, tz):
    """__all_sync over each warp (32 consecutive lanes tx = 0..31)."""
    key = np.stack([bx, by, bz, ty, tz], -1)
    _, inv = np.unique(key, axis=0, return_inverse=True)
    allw = np.ones(inv.max() + 1, dtype=bool)
    np.logical_and.at(allw, inv.ravel(), pred)
    return allw[inv.ravel()]


def check_vec(lo_elem, n, row_start, pitch, size):
    """A vector of n elements at lo_elem stays in its row and its buffer."""
    assert np.all(lo_elem >= 0) and np.all(lo_elem + n <= size)
    col = lo_elem - row_start
    assert np.all(col >= 0) and np.all(col + n <= pitch)


# ------------------------------------------------------------- thermal ----

def column_launch(nx, ny, nz, esize, rows):
    W = 4 if nz > 1 else VEC[esize]
    by_ = max(1, min(rows, 8))
    chunks = -(-nz // 8) if nz > 8 else 1
    return W, (-(-nx // (32 * W)), -(-ny // by_), chunks), (32, by_, 1)


@pytest.mark.parametrize("nx,ny,nz", [(130, 17, 1), (37, 29, 1), (5, 1, 1), (257, 66, 1), (33, 21, 5),
                                      (67, 13, 4), (45, 10, 8), (140, 6, 2), (70, 11, 24), (36, 9, 19),
                                      (130, 9, 17), (3, 2, 2), (512, 16, 8)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("rows", [1, 3, 8])
def test_column_kernel_addresses(nx, ny, nz, esize, rows):
    W, grid, block = column_launch(nx, ny, nz, esize, rows)
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    deep = nz > 8
    nzm = 8 if nz > 1 else 1
    exact = (nz == 1) or (nz in (2, 4, 8)) or (deep and nz % 8 == 0)
    if nz > 1 and nz in (2, 4):
        nzm = nz
    bx, by, bz, lane, ty, tz = threads(grid, block)
    x0 = (bx * 32 + lane) * W
    y = by * block[1] + ty
    z0 = bz * 8 if deep else np.zeros_like(bz)
    full_x = warp_all(x0 + W <= nx, bx, by, bz, ty, tz)
    fast = full_x & (y < ny)
    xc = np.where(fast, x0, np.minimum(x0, (nx - 1) // W * W))
    yc = np.where(fast, y, np.minimum(y, ny - 1))
    dn = np.where(yc > 0, -pitch, 0)
    ds = np.where(yc + 1 < ny, pitch, 0)
    dedge = np.where(lane == 0, np.where(xc > 0, -1, 0), np.minimum(W, nx - 1 - xc))
    nzl = np.full_like(z0, nzm) if exact else (np.minimum(8, nz - z0) if deep else np.full_like(z0, nz))
    assert np.all(nzl >= 1)
    covered = np.zeros(size, dtype=np.int64)
    for z in range(nzm):
        pz = z0 + (z if exact else np.minimum(z, nzl - 1))
        assert np.all(pz < nz)
        for d in (0, dn, ds):
            base = pz * plane + yc * pitch + xc + d
            check_vec(base, W, pz * plane + (yc * pitch + d), pitch, size)
        edge = pz * plane + yc * pitch + xc + dedge
        e = (lane == 0) | (lane == 31)
        check_vec(edge[e], 1, (pz * plane + yc * pitch)[e], pitch, size)
        # stores of the active threads (the update of plane z0 + z)
        act = (x0 < nx) & (y < ny) & (z < nzl)
        nv = np.where(full_x, W, np.minimum(W, nx - x0))
        s0 = (z0 + z) * plane + y * pitch + x0
        check_vec(s0[act], nv[act], ((z0 + z) * plane + y * pitch)[act], pitch, size)
        for k in range(W):
            m = act & (k < nv)
            np.add.at(covered, s0[m] + k, 1)
    if deep:
        for pz in (np.maximum(z0 - 1, 0), np.minimum(z0 + nzl, nz - 1)):
            check_vec(pz * plane + yc * pitch + xc, W, pz * plane + yc * pitch, pitch, size)
    check_vec(yc * pitch + xc, W, yc * pitch, pitch, ny * pitch)  # the P row
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)
    assert covered.max() <= 1


@pytest.mark.parametrize("nx,ny", [(300, 37), (96, 64), (77, 45), (500, 130), (3, 2), (1, 9), (130, 17)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("depth", [2, 4])
@pytest.mark.parametrize("block_x", [32, 64, 256])
def test_temporal_column_kernel_addresses(nx, ny, esize, depth, block_x):
    V = VEC[esize]
    R = 4 if V == 4 else 2
    BY = max(1, min(block_x // 32, 8))
    grid = (-(-nx // (30 * V)), -(-ny // (R * BY)), 1)
    pitch = pitch_of(nx, esize)
    size = pitch * ny
    bx, by, bz, lane, ty, tz = threads(grid, (32, BY, 1))
    xs = bx * 30 * V - V
    x0 = xs + lane * V
    y0 = (by * BY + ty) * R
    xc = np.minimum(np.maximum(x0, 0), (nx - 1) // V * V)
    NR = R + 2 * depth
    for k in range(NR):
        yk = np.clip(y0 - depth + k, 0, ny - 1)
        check_vec(yk * pitch + xc, V, yk * pitch, pitch, size)
    covered = np.zeros(size, dtype=np.int64)
    st = (lane >= 1) & (lane <= 30) & (x0 < nx)
    nv = np.minimum(V, nx - x0)
    for j in range(depth, depth + R):
        yg = y0 - depth + j
        m = st & (yg < ny)
        check_vec((yg * pitch + x0)[m], nv[m], (yg * pitch)[m], pitch, size)
        for k in range(V):
            mm = m & (k < nv)
            np.add.at(covered, (yg * pitch + x0)[mm] + k, 1)
    cells = np.zeros((ny, pitch), dtype=bool)
    cells[:, :nx] = True
    assert np.array_equal(covered.reshape(ny, pitch) == 1, cells)


# ---------------------------------------------------------------- FDTD ----

@pytest.mark.parametrize("N", [9, 16, 37, 128, 130])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("rows", [1, 2, 8])
def test_fdtd_column_kernel_addresses(N, esize, rows):
    V = 4
    M = N + 1
    aln = N % (32 * V) == 0
    pitch = pitch_of(M, esize)
    plane = pitch * M
    size = plane * M
    by_ = max(1, min(rows, 8))
    bz_ = max(1, 8 // by_)
    span = N if aln else M
    grid = (-(-span // (32 * V)), -(-M // by_), -(-M // bz_))
    bx, by, bz, lane, ty, tz = threads(grid, (32, by_, bz_))
    i0 = (bx * 32 + lane) * V
    j = by * by_ + ty
    k = bz * bz_ + tz
    in_x = np.ones_like(i0, dtype=bool) if aln else warp_all(i0 + V <= N, bx, by, bz, ty, tz)
    for half in ("H", "E"):
        if half == "H":
            fast = in_x & (j < N) & (k < N)
        else:
            fast = in_x & (j >= 1) & (j <= N - 1) & (k >= 1) & (k <= N - 1)
        act = fast | ((i0 < M) & (j < M) & (k < M))
        o = k * plane + j * pitch + i0
        row = k * plane + j * pitch
        nv = np.where(fast, V, np.minimum(V, M - i0))
        a = act
        check_vec(o[a], nv[a], row[a], pitch, size)  # own vectors (loads and stores)
        if half == "H":
            for d, cond in ((plane, k + 1 < M), (pitch, j + 1 < M)):
                m = a & (fast | cond)
                check_vec((o + d)[m], nv[m], (row + d)[m], pitch, size)
            m = a & (lane == 31) & (fast | (i0 + V < M))
            check_vec((o + V)[m], 1, row[m], pitch, size)
            if aln:  # lane 31's i = N cell: Ez at j+1, Ey at k+1, Hx
                m = fast & (lane == 31)
                assert np.all(i0[m] + V == N)
                for d in (pitch, plane, 0):
                    check_vec((o + d + V)[m], 1, (row + d)[m], pitch, size)
        else:
            for d, cond in ((-plane, k >= 1), (-pitch, j >= 1)):
                m = a & (fast | cond)
                check_vec((o + d)[m], nv[m], (row + d)[m], pitch, size)
            dw = np.where(fast, np.where(i0 > 0, -1, 0), -1)
            m = a & (lane == 0) & (fast | (i0 >= 1))
            check_vec((o + dw)[m], 1, row[m], pitch, size)
    # every (i, j, k) of the (N+1)^3 arrays is some thread's own cell, or
    # (aligned layout) lane 31's extra cell i = N
    owned = np.zeros(size, dtype=np.int64)
    act = (i0 < M) & (j < M) & (k < M)
    nv = np.minimum(V, M - i0)
    o = k * plane + j * pitch + i0
    for c in range(V):
        m = act & (c < nv)
        np.add.at(owned, o[m] + c, 1)
    if aln:
        m = act & (lane == 31) & (i0 + V == N)
        np.add.at(owned, o[m] + V, 1)
    cells = np.zeros((M, M, pitch), dtype=bool)
    cells[:, :, :M] = True
    assert np.array_equal(owned.reshape(M, M, pitch) == 1, cells)
