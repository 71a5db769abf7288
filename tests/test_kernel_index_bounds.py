"""CPU re-trace of the kernels' index arithmetic: the COLUMN kernels (thermal
depth 1 in 2D, thin and chunked deep stacks; thermal depth 2 and 4 in 2D;
the FDTD H and E kernels in the aligned and general layouts), COLUMN_SMEM
(its shared slab of neighbour rows), the FDTD k-march kernels, the MARCH
kernel (2D and 3D, with its shared-memory plane slab), the WAVE kernel
(depths 1, 2 and 4, with its 3D level buffers), and the work items of the
multi-instance kernel (host table, persistent loop, binary search, tile
stores).  For every thread of every block of the launch the library makes,
every global load and store must lie inside its buffer and inside its row
(the pitch), every shared-memory access inside the launch's allocation, and
the stores of a launch must cover every cell of the field exactly once.
The 3D depth-t COLUMN kernel (one cell a lane, every plane of the column)
and the z-marching depth-2 kernel of deep stacks are re-traced the same way,
and so are the fused FDTD step (H and E in one launch, out of place; its
column form and its k march) and the STREAM kernel (its tensor-copy boxes, shared-memory ring and stores).
The formulas restate the kernels' address computations (csrc/heat.cu,
csrc/fdtd.cu, csrc/multi.cu) for ragged shapes, so that a change to either
is checked here before it runs on a GPU."""
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


def every_block_stores(stored, bx, by, bz):
    """No block of the launch is empty (the grid is not over-sized)."""
    key = (bx * 65536 + by) * 65536 + bz
    assert np.array_equal(np.unique(key[stored]), np.unique(key))


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


@pytest.mark.parametrize("nx,ny,nz", [(512, 24, 8), (97, 41, 8), (40, 33, 7), (30, 9, 4), (29, 5, 3), (1, 9, 2),
                                      (57, 1, 8), (3, 2, 5), (2, 3, 1)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("depth,rows", [(2, 4), (2, 2), (4, 4)])
@pytest.mark.parametrize("block_x", [32, 128, 256])
def test_temporal_column3_kernel_addresses(nx, ny, nz, esize, depth, rows, block_x):
    # one cell a lane, 32 - 2t stored lanes a warp, R rows a warp row (4 at
    # depth 2 unless plan.rows is 2; 2 at depth 4), loads of rows y0-t ..
    # y0+R+t-1 of every plane at clamped coordinates; EXACT kernels hold nz
    # planes (nz 4 or 8), the others eight
    R = 4 if (depth == 2 and rows != 2) else 2
    BY = max(1, min(block_x // 32, 8))
    span = 32 - 2 * depth
    grid = (-(-nx // span), -(-ny // (R * BY)), 1)
    NZM = nz if nz in (4, 8) else 8
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    bx, by, bz, lane, ty, tz = threads(grid, (32, BY, 1))
    xs = bx * span - depth
    x = xs + lane
    xc = np.minimum(np.maximum(x, 0), nx - 1)
    y0 = (by * BY + ty) * R
    NR = R + 2 * depth
    for k in range(NR):
        yk = np.clip(y0 - depth + k, 0, ny - 1)
        for z in range(NZM):
            zc = min(z, nz - 1)
            check_vec(zc * plane + yk * pitch + xc, 1, zc * plane + yk * pitch, pitch, size)
    for k in range(1, NR - 1):  # P rows (one plane)
        yk = np.clip(y0 - depth + k, 0, ny - 1)
        check_vec(yk * pitch + xc, 1, yk * pitch, pitch, pitch * ny)
    covered = np.zeros(size, dtype=np.int64)
    st = (lane >= depth) & (lane < 32 - depth) & (x < nx)
    for j in range(depth, depth + R):
        yg = y0 - depth + j
        m = st & (yg < ny)
        for z in range(min(NZM, nz)):
            addr = (z * plane + yg * pitch + x)[m]
            check_vec(addr, 1, (z * plane + yg * pitch)[m], pitch, size)
            np.add.at(covered, addr, 1)
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)
    assert covered.max() <= 1
    every_block_stores(st & (y0 < ny), bx, by, bz)


@pytest.mark.parametrize("nx,ny,nz", [(256, 24, 40), (97, 41, 9), (61, 9, 17), (5, 3, 33), (121, 1, 12), (2, 7, 10)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("block_x", [32, 128, 256])
@pytest.mark.parametrize("chunk", [1, 5, 32])
def test_zmarch2_kernel_addresses(nx, ny, nz, esize, block_x, chunk):
    # deep stacks at depth 2: two cells a lane (pairs at even x, clamped to
    # the last pair that starts inside the row), lanes 1..30 store, four rows
    # a warp, blocks of BY <= 4 warps marching `chunk` planes; level-0 planes
    # z0-2 .. z1+1 are loaded where inside the stack, rows clamped
    W, R = 2, 4
    BY = max(1, min(block_x // 32, 4))
    grid = (-(-nx // (30 * W)), -(-ny // (R * BY)), -(-nz // chunk))
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    bx, by, bz, lane, ty, tz = threads(grid, (32, BY, 1))
    x0 = bx * 30 * W - W + lane * W
    xc = np.minimum(np.maximum(x0, 0), (nx - 1) // W * W)
    y0 = (by * BY + ty) * R
    z0 = bz * chunk
    z1 = np.minimum(z0 + chunk, nz)
    for dz in range(-2, chunk + 2):
        z = z0 + dz
        m = (z >= 0) & (z < nz) & (z <= z1 + 1)
        for k in range(R + 4):
            yk = np.clip(y0 - 2 + k, 0, ny - 1)
            check_vec((z * plane + yk * pitch + xc)[m], W, (z * plane + yk * pitch)[m], pitch, size)
    for yg in range(-1, R + 5):  # P rows of plane 0 (clamped)
        yk = np.clip(y0 + yg, 0, ny - 1)
        check_vec(yk * pitch + xc, W, yk * pitch, pitch, pitch * ny)
    covered = np.zeros(size, dtype=np.int64)
    st = (lane >= 1) & (lane <= 30) & (x0 < nx)
    nv = np.minimum(W, nx - x0)
    for dz in range(chunk):
        z = z0 + dz
        for i in range(R):
            yg = y0 + i
            m = st & (z < z1) & (yg < ny)
            addr = (z * plane + yg * pitch + x0)[m]
            check_vec(addr, nv[m], (z * plane + yg * pitch)[m], pitch, size)
            for c in range(W):
                mc = m & (c < nv)
                np.add.at(covered, (z * plane + yg * pitch + x0)[mc] + c, 1)
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)
    every_block_stores(st & (y0 < ny) & (z0 < nz), bx, by, bz)


@pytest.mark.parametrize("nx,ny,nz", [(256, 24, 40), (97, 41, 9), (130, 9, 17), (5, 3, 33), (121, 1, 12),
                                      (2, 7, 10), (300, 30, 3), (128, 40, 1)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("block_x", [256, 512])
@pytest.mark.parametrize("chunk", [1, 5, 32])
def test_stream2_kernel_addresses(nx, ny, nz, esize, block_x, chunk):
    # the STREAM kernel (3D, depth 2): tiles of 128 x (2W - 2) stored cells,
    # W compute warps (four cells a lane at level-1 rows 2w, 2w+1), one
    # halo warp; stage boxes of (128 + 2 PX) x (2W + 2) elements from
    # (x0 - PX, y0 - 2, plane); a ring of 6 stages refilled after step r
    # with plane r - 2 + 6; two level-1 planes
    W = 16 if block_x >= 512 else 8
    R = 2
    PX = 16 // esize
    BWC = 128 + 2 * PX
    L1R, S = W * R, 6
    BR = L1R + 2
    stage_bytes = -(-(BR * BWC * esize) // 128) * 128
    smem = S * stage_bytes + 2 * L1R * BWC * 4 + 8 * S  # stages, two level-1 planes, mbarriers
    assert smem <= 227 * 1024 and (W > 8 or 2 * smem <= 228 * 1024)
    assert BWC <= 256 and BR <= 256 and (BWC * esize) % 16 == 0 and BR * BWC * esize < (1 << 20)
    assert (S * stage_bytes) % 16 == 0 and (S * stage_bytes + 2 * L1R * BWC * 4) % 8 == 0
    grid = (-(-nx // 128), -(-ny // (L1R - 2)), -(-nz // chunk))
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    bx, by, bz = [a.ravel() for a in np.meshgrid(*[np.arange(n) for n in grid], indexing="ij")]
    x0, y0, z0 = bx * 128, by * (L1R - 2), bz * chunk
    z1 = np.minimum(z0 + chunk, nz)
    assert np.all(((x0 - PX) * esize) % 16 == 0)  # the box's x coordinate: 16-byte aligned
    assert np.all(z0 < nz)  # no empty block along z
    # the ring: simulate the copies and waits of one block (n0 depends only on the chunk)
    for n0 in np.unique(z1 - z0 + 4):
        resident = {}
        fills = [0] * S
        for q in range(min(S, n0)):
            resident[q % S] = q
        issued = min(S, n0)
        for r in range(n0):
            assert resident[r % S] == r and (r // S) & 1 == (fills[r % S]) & 1  # waited plane and phase
            fills[r % S] += 1
            if r >= 2:
                for q in (r - 2, r - 1, r):  # the planes level 1 reads
                    assert resident[q % S] == q
            if r >= 2 and issued < n0:
                assert issued == r - 2 + S
                resident[issued % S] = issued
                issued += 1
        assert issued == n0
    # per thread: stage reads (compute warps: rows i..i+2 of mid, row i+1 of lo/hi, cols PX+4l..+3 and the
    # edge columns PX-1, PX+128; halo warp: rows i..i+2, cols PX-2..PX and PX+127..PX+129), L1 reads
    lane = np.arange(32)
    cols = PX + 4 * lane
    assert cols.min() >= 0 and (cols + 3).max() < BWC and PX - 1 >= 0 and PX + 128 < BWC
    for w in range(W):
        i0 = R * w
        assert 0 <= i0 and i0 + R + 1 < BR  # level 1: stage rows i0 .. i0 + R + 1
        assert 0 <= i0 - 1 or w == 0  # level 2: level-1 rows i0 - 1 (not for the block's first row) ..
        assert i0 + R < L1R or w == W - 1  # .. i0 + R (not for its last)
    for i in range(L1R):  # the halo warp: stage rows i .. i + 2, columns around PX - 1 and PX + 128
        assert 0 <= i and i + 2 < BR
        for cc in (PX - 1, PX + 128):
            assert 0 <= cc - 1 and cc + 1 < BWC
    # stores of level 2: rows i in [1, L1R-2] (y = y0 - 1 + i < ny), lanes with x = x0 + 4 lane < nx,
    # planes [z0, z1); P reads at clamped coordinates
    covered = np.zeros(size, dtype=np.int64)
    for w in range(W):
        for k in range(R):
            i = w * R + k
            if not 1 <= i <= L1R - 2:
                continue
            y = y0 - 1 + i
            for l in range(32):
                x = x0 + 4 * l
                nv = np.minimum(4, nx - x)
                for dz in range(chunk):
                    z = z0 + dz
                    m = (y < ny) & (x < nx) & (z < z1)
                    addr = (z * plane + y * pitch + x)[m]
                    check_vec(addr, nv[m], (z * plane + y * pitch)[m], pitch, size)
                    for c in range(4):
                        mc = m & (c < nv)
                        np.add.at(covered, (z * plane + y * pitch + x)[mc] + c, 1)
            yc = np.clip(y, 0, ny - 1)
            assert np.all(yc * pitch + np.clip(x0 + 4 * 31 + 3, 0, nx - 1) < pitch * ny)
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)
    # every block stores something (the grid is not over-sized)
    assert np.all((x0 < nx) & (y0 < ny) & (z0 < nz))


# ---------------------------------------------------------------- FDTD ----

@pytest.mark.parametrize("N", [9, 16, 37, 128, 130, 256])
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
            if aln:  # the i = N cell of the last block's lane 31: Ez at j+1, Ey at k+1, Hx
                m = fast & (lane == 31) & (i0 + V == N)
                assert m.sum() == N * N  # one per (j, k) of the FAST H body
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


@pytest.mark.parametrize("N,Nk", [(9, 9), (16, 16), (37, 37), (128, 128), (130, 130), (64, 17), (128, 33), (16, 1),
                                  (256, 9)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("rows", [1, 2, 8])
def test_fdtd_fused_kernel_addresses(N, Nk, esize, rows):
    # the fused step: own vectors and the j+1, k+1, j-1, k-1, j-1&k+1,
    # k-1&j+1 vectors at offsets that collapse to 0 where they would leave
    # the arrays (and for threads past them), lane 31's i+1 scalars, lane
    # 0's i-1 scalars, the aligned layout's i = N cell; stores of all six
    # components cover every element of the written set once
    V = 4
    M, Mk = N + 1, Nk + 1
    aln = N % (32 * V) == 0
    pitch = pitch_of(M, esize)
    plane = pitch * M
    size = plane * Mk
    by_ = max(1, min(rows, 8))
    bz_ = max(1, 8 // by_)
    span = N if aln else M
    grid = (-(-span // (32 * V)), -(-M // by_), -(-Mk // bz_))
    bx, by, bz, lane, ty, tz = threads(grid, (32, by_, bz_))
    i0 = (bx * 32 + lane) * V
    j = by * by_ + ty
    k = bz * bz_ + tz
    in_x = np.ones_like(i0, dtype=bool) if aln else warp_all(i0 + V <= N, bx, by, bz, ty, tz)
    fast = in_x & (j >= 1) & (j <= N - 1) & (k >= 1) & (k <= Nk - 1)
    act = fast | ((i0 < M) & (j < M) & (k < Mk))
    o = np.where(act, k * plane + j * pitch + i0, 0)
    row = np.where(act, k * plane + j * pitch, 0)
    dj1 = np.where(fast | (act & (j + 1 < M)), pitch, 0)
    dk1 = np.where(fast | (act & (k + 1 < Mk)), plane, 0)
    djm = np.where(fast | (act & (j >= 1)), -pitch, 0)
    dkm = np.where(fast | (act & (k >= 1)), -plane, 0)
    # vector loads of every thread (inactive ones at offset 0)
    for d in (0, dk1, dj1, djm, djm + dk1, dkm, dkm + dj1):
        check_vec(o + d, V, row + d, pitch, size)
    has_r = (lane == 31) & (fast | (act & (i0 + V < M)))
    for d in (0, djm, dkm):
        check_vec((o + d + V)[has_r], 1, (row + d)[has_r], pitch, size)
    if aln:
        xr = has_r & (i0 + V == N)
        for d in (dj1, dk1):
            check_vec((o + d + V)[xr], 1, (row + d)[xr], pitch, size)
    m = (lane == 0) & (i0 >= 1) & act
    for d in (0, dj1, dk1):
        check_vec((o + d - 1)[m], 1, (row + d)[m], pitch, size)
    # stores: every element of the M x M x Mk arrays once
    owned = np.zeros(size, dtype=np.int64)
    nv = np.where(fast, V, np.minimum(V, M - i0))
    for c in range(V):
        mm = act & (c < nv)
        np.add.at(owned, o[mm] + c, 1)
    if aln:  # the i = N cell: the last block's lane 31 only
        mm = act & (lane == 31) & (i0 + V == N)
        np.add.at(owned, o[mm] + V, 1)
    cells = np.zeros((Mk, M, pitch), dtype=bool)
    cells[:, :, :M] = True
    assert np.array_equal(owned.reshape(Mk, M, pitch) == 1, cells)


@pytest.mark.parametrize("N,Nk", [(9, 9), (16, 16), (37, 37), (128, 128), (130, 130), (64, 17), (128, 33), (16, 1),
                                  (256, 9)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("rows,kmarch", [(1, 1), (2, 5), (8, 16), (4, 300)])
def test_fdtd_fused_march_kernel_addresses(N, Nk, esize, rows, kmarch):
    # the fused step marching kmarch planes in k (block 32 x rows, one warp
    # a row j): the prologue's own and j-1 vectors at k0 and, above the
    # bottom wall, the plane k0-1 vectors (and lane 31's i+1 scalar); per
    # plane the own, k+1, j+1, j-1 and j-1&k+1 vectors at offsets that
    # collapse to 0 where they would leave the arrays, lanes past the
    # arrays loading at the start of their row; lane 31's i+1 scalars,
    # lane 0's i-1 scalars, the aligned layout's i = N cell; stores of all
    # six components cover every element of the written set once.  In media
    # the uint8 ids are read at the own, j-1 and k0-1 vectors' offsets and
    # the i-1 and i = N scalars' (the map has the fields' pitch in
    # elements), so the same checks cover them.
    V = 4
    M, Mk = N + 1, Nk + 1
    aln = N % (32 * V) == 0
    pitch = pitch_of(M, esize)
    plane = pitch * M
    size = plane * Mk
    by_ = max(1, min(rows, 8))
    span = N if aln else M
    grid = (-(-span // (32 * V)), -(-M // by_), -(-Mk // kmarch))
    bx, by, bz, lane, ty, _ = threads(grid, (32, by_, 1))
    i0 = (bx * 32 + lane) * V
    j = by * by_ + ty
    k0 = bz * kmarch
    k1 = np.minimum(k0 + kmarch, Mk)
    live = j < M  # warps past the last row return at once
    act_i = np.ones_like(i0, dtype=bool) if aln else (i0 < M)
    in_x = np.ones_like(i0, dtype=bool) if aln else warp_all(i0 + V <= N, bx, by, bz, ty, np.zeros_like(ty))
    fast_j = in_x & (j >= 1) & (j <= N - 1)
    # prologue
    o = k0 * plane + j * pitch + np.where(act_i, i0, 0)
    row = k0 * plane + j * pitch
    djm = np.where(j >= 1, -pitch, 0)
    dj1 = np.where(j + 1 < M, pitch, 0)
    m = live
    for d in (0, djm):
        check_vec((o + d)[m], V, (row + d)[m], pitch, size)
    m = live & (k0 >= 1)
    for d in (-plane, -plane + dj1):
        check_vec((o + d)[m], V, (row + d)[m], pitch, size)
    m = m & (lane == 31) & act_i & (i0 + V < M)
    check_vec((o - plane + V)[m], 1, (row - plane)[m], pitch, size)
    owned = np.zeros(size, dtype=np.int64)
    for p in range(min(kmarch, Mk)):
        k = k0 + p
        m0 = live & (k < k1)
        fast = fast_j & (k >= 1) & (k <= Nk - 1)
        dj1 = np.where(fast | (j + 1 < M), pitch, 0)
        dk1 = np.where(fast | (k + 1 < Mk), plane, 0)
        djm = np.where(fast | (j >= 1), -pitch, 0)
        act = fast | act_i
        o = k * plane + j * pitch + np.where(act, i0, 0)
        row = k * plane + j * pitch
        for d in (0, dk1, dj1, djm, djm + dk1):
            check_vec((o + d)[m0], V, (row + d)[m0], pitch, size)
        has_r = m0 & (lane == 31) & (fast | (act_i & (i0 + V < M)))
        for d in (0, djm):
            check_vec((o + d + V)[has_r], 1, (row + d)[has_r], pitch, size)
        if aln:
            xr = has_r & (i0 + V == N)
            for d in (dj1, dk1):
                check_vec((o + d + V)[xr], 1, (row + d)[xr], pitch, size)
        ml = m0 & (lane == 0) & (i0 >= 1) & act
        for d in (0, dj1, dk1):
            check_vec((o + d - 1)[ml], 1, (row + d)[ml], pitch, size)
        ms = m0 & act
        nv = np.where(fast, V, np.minimum(V, M - i0))
        for c in range(V):
            mm = ms & (c < nv)
            np.add.at(owned, o[mm] + c, 1)
        if aln:  # the i = N cell: the last block's lane 31 only
            mm = ms & (lane == 31) & (i0 + V == N)
            check_vec((o + V)[mm], 1, row[mm], pitch, size)
            np.add.at(owned, o[mm] + V, 1)
    cells = np.zeros((Mk, M, pitch), dtype=bool)
    cells[:, :, :M] = True
    assert np.array_equal(owned.reshape(Mk, M, pitch) == 1, cells)
    # no block is empty
    assert np.all(((by * by_) < M) & (k0 < Mk) & (bx * 32 * V < span))


# ---------------------------------------------------- MARCH and WAVE ----

@pytest.mark.parametrize("nx,ny,nz", [(300, 37, 1), (77, 45, 1), (3, 2, 1), (513, 9, 1), (130, 17, 3),
                                      (64, 10, 8), (90, 7, 16), (33, 5, 20), (5, 4, 2)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("block_x,rows", [(32, 4), (64, 1), (128, 7), (256, 16)])
def test_march_kernel_addresses(nx, ny, nz, esize, block_x, rows):
    # heat_march_tile: thread (tx, tz) owns V cells at x0 = (bx BX + tx) V of
    # plane z = bz ZB + tz and marches rows y0 .. y1-1 of its block's tile
    V = VEC[esize]
    is3d = nz > 1
    zb = min(min(nz, 16), max(1, 512 // block_x)) if is3d else 1
    assert block_x * zb <= 512  # __launch_bounds__(512)
    grid = (-(-nx // (block_x * V)), -(-ny // rows), -(-nz // zb) if is3d else 1)
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    bx, by, bz, tx, tz, _ = threads(grid, (block_x, zb, 1))
    x0 = (bx * block_x + tx) * V
    z0 = bz * zb
    z = z0 + tz
    y0 = by * rows
    y1 = np.minimum(y0 + rows, ny)
    act = (x0 < nx) & (z < nz)
    has_p = (z == 0) if is3d else np.ones_like(act)
    dn = is3d & (tz == 0) & (z0 > 0) & (x0 < nx)
    up = is3d & (tz == zb - 1) & (z0 + zb < nz) & (x0 < nx)
    lane = tx & 31
    covered = np.zeros(size, dtype=np.int64)
    stored = np.zeros_like(act)
    for k in range(-1, rows + 1):  # rows y0-1 .. y0+rows of the tile
        y = y0 + k
        inrow = (y >= 0) & (y < ny) & (y <= y1)
        m = act & inrow
        check_vec((z * plane + y * pitch + x0)[m], V, (z * plane + y * pitch)[m], pitch, size)
        for halo, dz in ((dn, -1), (up, 1)):
            mh = halo & (y >= y0) & (y < y1)
            check_vec(((z + dz) * plane + y * pitch + x0)[mh], V, ((z + dz) * plane + y * pitch)[mh], pitch, size)
        tile = (y >= y0) & (y < y1)
        mp = act & has_p & tile
        check_vec((y * pitch + x0)[mp], V, (y * pitch)[mp], pitch, ny * pitch)
        for cond, off in (((lane == 0) & (x0 > 0), -1), ((lane == 31) & (x0 + V < nx), V)):
            ms = act & tile & cond
            check_vec((z * plane + y * pitch + x0 + off)[ms], 1, (z * plane + y * pitch)[ms], pitch, size)
        # stores of row y
        ms = act & tile
        stored |= ms
        nv = np.minimum(V, nx - x0)
        check_vec((z * plane + y * pitch + x0)[ms], nv[ms], (z * plane + y * pitch)[ms], pitch, size)
        for c in range(V):
            mm = ms & (c < nv)
            np.add.at(covered, (z * plane + y * pitch + x0)[mm] + c, 1)
    if is3d:  # the shared slab [2][ZB+2][BX V]: rows tz, tz+1, tz+2, 0 and ZB+1
        rowlen = block_x * V
        for r in (tz, tz + 1, tz + 2, np.zeros_like(tz), np.full_like(tz, zb + 1)):
            off = (zb + 2) * rowlen + r * rowlen + tx * V
            assert np.all(off + V <= 2 * (zb + 2) * rowlen)
    every_block_stores(stored, bx, by, bz)
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)


@pytest.mark.parametrize("nx,ny,nz", [(300, 37, 1), (77, 45, 1), (3, 2, 1), (130, 17, 1), (500, 9, 1),
                                      (131, 19, 3), (64, 10, 8), (250, 7, 16), (5, 5, 2)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("depth", [1, 2, 4])
@pytest.mark.parametrize("block_x,rows", [(64, 4), (128, 32), (32, 1), (96, 7)])
def test_wave_kernel_addresses(nx, ny, nz, esize, depth, block_x, rows):
    # heat_wave_kernel: warps of 32 vectors at x0 = bx 30V - V + lane V
    # (lanes 0 and 31 are halo lanes), marching level-0 rows y0-T ..
    # y0+R+T-1 and storing level T's rows y0 .. y0+R-1 from lanes 1..30
    V = VEC[esize]
    is3d = nz > 1
    stride = 30 * V
    wb = nz if is3d else max(1, block_x // 32)
    ry = rows if is3d else rows * wb
    assert 32 * wb <= 512  # __launch_bounds__(512)
    grid = (-(-nx // stride), -(-ny // ry), 1)
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    bx, by, bz, lane, ty, _ = threads(grid, (32, wb, 1))
    x0 = bx * stride - V + lane * V
    zz = ty if is3d else np.zeros_like(ty)
    y0 = by * rows if is3d else (by * wb + ty) * rows
    has_p = (zz == 0) if is3d else np.ones_like(lane, dtype=bool)
    ld_ok = (x0 >= 0) & (x0 < nx)
    st_lane = (lane >= 1) & (lane <= 30) & (x0 < nx)
    nsteps = rows + 2 * depth
    covered = np.zeros(size, dtype=np.int64)
    nv = np.minimum(V, nx - x0)
    stored = np.zeros_like(ld_ok)
    for j in range(nsteps):
        r = y0 - depth + j
        m = ld_ok & (r >= 0) & (r < ny)
        check_vec((zz * plane + r * pitch + x0)[m], V, (zz * plane + r * pitch)[m], pitch, size)
        mp = m & has_p
        check_vec((r * pitch + x0)[mp], V, (r * pitch)[mp], pitch, ny * pitch)
        q = r - depth  # the row level T computes at this march step
        ms = st_lane & (q >= y0) & (q < y0 + rows) & (q < ny)
        stored |= ms
        check_vec((zz * plane + q * pitch + x0)[ms], nv[ms], (zz * plane + q * pitch)[ms], pitch, size)
        for c in range(V):
            mm = ms & (c < nv)
            np.add.at(covered, (zz * plane + q * pitch + x0)[mm] + c, 1)
    if is3d:  # [2][T][nz][32 V] floats: writes at level s < T, reads at s-1 of planes tz +- 1
        rowlen = 32 * V
        total = 2 * depth * nz * rowlen
        assert total * 4 == 2 * depth * nz * 32 * V * 4 <= 227 * 1024
        for buf in (0, 1):
            for s in range(depth):
                off = buf * depth * nz * rowlen + lane * V + (s * nz + zz) * rowlen
                assert np.all(off >= 0) and np.all(off + V <= total)
            for s in range(1, depth + 1):
                base = buf * depth * nz * rowlen + lane * V + (s - 1) * nz * rowlen
                for zn, ok in ((zz - 1, zz > 0), (zz + 1, zz + 1 < nz)):
                    off = (base + zn * rowlen)[ok]
                    assert np.all(off >= 0) and np.all(off + V <= total)
    every_block_stores(stored, bx, by, bz)
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)


# ------------------------------------------------- instance batches ----

# widths 125 and 250 need one more tile of 30 vectors than of 32 (f32, bf16)
MULTI_DIMS = [(130, 17), (5, 9), (64, 64), (200, 3), (1, 1), (77, 120), (300, 41), (64, 64), (125, 13), (250, 6)]


def multi_table(dims, esize, kind, block_x, rows):
    """The descriptor table build_table makes: instances largest first
    (stable), tiles of `span` cells by `item_rows` rows, first_item the
    running sum of the items before."""
    V = VEC[esize]
    col = kind != 0
    span = (30 * V if kind > 1 else 32 * V) if col else block_x * V
    item_rows = rows * (4 if V == 4 else 2) if kind > 1 else rows
    order = sorted(range(len(dims)), key=lambda i: -dims[i][0] * dims[i][1])  # sorted() is stable
    table, item = [], 0
    for i in order:
        nx, ny = dims[i]
        ntx, nty = -(-nx // span), -(-ny // item_rows)
        table.append(dict(inst=i, nx=nx, ny=ny, first=item, n=ntx * nty, ntx=ntx))
        item += ntx * nty
    return table, item, span


def tile_stores(kind, esize, nx, ny, tx_, ty_, block_x, rows):
    """(x0, y, n_valid) of every store the tile (tx_, ty_) makes."""
    V = VEC[esize]
    out = []
    if kind == 0:  # MARCH tile: block_x threads, rows y0 .. y1-1
        for t in range(block_x):
            x0 = (tx_ * block_x + t) * V
            if x0 < nx:
                out += [(x0, y, min(V, nx - x0)) for y in range(ty_ * rows, min(ty_ * rows + rows, ny))]
    elif kind == 1:  # COLUMN tile, depth 1: (32, rows) threads, one row each
        for ty in range(rows):
            y = ty_ * rows + ty
            for lane in range(32):
                x0 = (tx_ * 32 + lane) * V
                if x0 < nx and y < ny:
                    out.append((x0, y, min(V, nx - x0)))
    else:  # COLUMN tile of temporal depth `kind`: R rows per warp row, lanes 1..30 store
        R = 4 if V == 4 else 2
        for ty in range(rows):
            y0 = (ty_ * rows + ty) * R
            for lane in range(1, 31):
                x0 = tx_ * 30 * V - V + lane * V
                if x0 < nx:
                    out += [(x0, y, min(V, nx - x0)) for y in range(y0, min(y0 + R, ny))]
    return out


@pytest.mark.parametrize("kind", [0, 1, 2, 4])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("blocks", [1, 7, 608])
@pytest.mark.parametrize("rev", [0, 1])
@pytest.mark.parametrize("block_x,rows", [(64, 4), (32, 1), (128, 3)])
def test_multi_items_cover_every_instance_once(kind, esize, blocks, rev, block_x, rows):
    # heat_multi_kernel: block b takes items b, b + grid, ... (last to first
    # on reversed launches), finds its instance by binary search on
    # first_item, and runs tile (item mod ntx, item div ntx) of it
    table, total, _ = multi_table(MULTI_DIMS, esize, kind, block_x, rows)
    grid = max(1, min(blocks, total))
    firsts = [d["first"] for d in table]
    seen = np.zeros(total, dtype=np.int64)
    cover = {d["inst"]: np.zeros((d["ny"], d["nx"]), dtype=np.int64) for d in table}
    for b in range(grid):
        for w0 in range(b, total, grid):
            w = total - 1 - w0 if rev else w0
            lo, hi = 0, len(table) - 1
            while lo < hi:
                mid = (lo + hi + 1) >> 1
                if firsts[mid] <= w:
                    lo = mid
                else:
                    hi = mid - 1
            d = table[lo]
            assert d["first"] <= w < d["first"] + d["n"], (w, lo)
            seen[w] += 1
            item = w - d["first"]
            for x0, y, nv in tile_stores(kind, esize, d["nx"], d["ny"], item % d["ntx"], item // d["ntx"],
                                         block_x, rows):
                assert 0 <= x0 and x0 + nv <= d["nx"] and 0 <= y < d["ny"]
                cover[d["inst"]][y, x0:x0 + nv] += 1
    assert np.all(seen == 1)
    for i, c in cover.items():
        assert np.all(c == 1), i


@pytest.mark.parametrize("N", [9, 16, 37, 64])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("block_x,kc", [(32, 1), (64, 4), (128, 16), (256, 3)])
def test_fdtd_kmarch_kernel_addresses(N, esize, block_x, kc):
    # fdtd_h/e_kernel: thread owns V cells along i at one j and marches
    # planes k0 .. k1-1 (kc per block); block (block_x, 256 / block_x)
    V = VEC[esize]
    M = N + 1
    pitch = pitch_of(M, esize)
    plane = pitch * M
    size = plane * M
    by_ = max(1, 256 // block_x)
    assert block_x * by_ <= 256  # __launch_bounds__(256)
    grid = (-(-M // (block_x * V)), -(-M // by_), -(-M // kc))
    bx, by, bz, tx, ty, _ = threads(grid, (block_x, by_, 1))
    i0 = (bx * block_x + tx) * V
    j = by * by_ + ty
    k0 = bz * kc
    lane = tx & 31
    act = (i0 < M) & (j < M)
    nv = np.minimum(V, M - i0)
    row = j * pitch
    owned = np.zeros(size, dtype=np.int64)
    stored = np.zeros_like(act)
    for dk in range(-1, kc + 1):
        k = k0 + dk
        o = k * plane + row + i0
        base = k * plane + row
        # H: own vectors at k (and k+1 / j+1 neighbours); E: own vectors at
        # k (and k-1 plane before the march, j-1 neighbours)
        mine = act & (k >= k0) & (k < np.minimum(k0 + kc, M))
        check_vec(o[mine], V, base[mine], pitch, size)
        mk1 = mine & (k + 1 < M)
        check_vec((o + plane)[mk1], V, (base + plane)[mk1], pitch, size)
        mj1 = mine & (j + 1 < M)
        check_vec((o + pitch)[mj1], V, (base + pitch)[mj1], pitch, size)
        mjm = mine & (j >= 1)
        check_vec((o - pitch)[mjm], V, (base - pitch)[mjm], pitch, size)
        mkm = act & (k == k0 - 1) & (k0 > 0)  # the E march's first k-1 plane
        check_vec(o[mkm], V, base[mkm], pitch, size)
        me = mine & (lane == 31) & (i0 + V < M)
        check_vec((o + V)[me], 1, base[me], pitch, size)
        mw = mine & (lane == 0) & (i0 >= 1)
        check_vec((o - 1)[mw], 1, base[mw], pitch, size)
        check_vec(o[mine], nv[mine], base[mine], pitch, size)  # stores
        stored |= mine
        for c in range(V):
            m = mine & (c < nv)
            np.add.at(owned, o[m] + c, 1)
    every_block_stores(stored, bx, by, bz)
    cells = np.zeros((M, M, pitch), dtype=bool)
    cells[:, :, :M] = True
    assert np.array_equal(owned.reshape(M, M, pitch) == 1, cells)


def _column_owner_cells(N, rows):
    """(i0, j, k, extra) of every active thread of a column E launch; extra
    marks lane 31 of the aligned layout, which also owns cell i0 + V."""
    V, M = 4, N + 1
    aln = N % (32 * V) == 0
    by_ = max(1, min(rows, 8))
    bz_ = max(1, 8 // by_)
    span = N if aln else M
    grid = (-(-span // (32 * V)), -(-M // by_), -(-M // bz_))
    bx, by, bz, lane, ty, tz = threads(grid, (32, by_, bz_))
    i0 = (bx * 32 + lane) * V
    j = by * by_ + ty
    k = bz * bz_ + tz
    act = (i0 < M) & (j < M) & (k < M)  # FAST threads are in range too
    return i0[act], j[act], k[act], (aln & (lane == 31))[act], V


def _kmarch_owner_cells(N, esize, block_x, kc):
    """(i0, j, k, extra) of every (active thread, marched plane) of a
    k-march E launch."""
    V, M = VEC[esize], N + 1
    by_ = max(1, 256 // block_x)
    grid = (-(-M // (block_x * V)), -(-M // by_), -(-M // kc))
    bx, by, bz, tx, ty, _ = threads(grid, (block_x, by_, 1))
    i0 = (bx * block_x + tx) * V
    j = by * by_ + ty
    k0 = bz * kc
    act = (i0 < M) & (j < M)
    out = [], [], []
    for dk in range(kc):
        m = act & (k0 + dk < M)
        out[0].append(i0[m])
        out[1].append(j[m])
        out[2].append((k0 + dk)[m])
    i0, j, k = (np.concatenate(v) for v in out)
    return i0, j, k, np.zeros_like(i0, dtype=bool), V


@pytest.mark.parametrize("N", [9, 37, 128, 130])
def test_fdtd_source_cell_has_one_owner(N):
    # the thread that owns the source cell adds the pulse and advances the
    # device step counter: exactly one thread of every E launch must own
    # each cell (si, sj, sk) in [0, N]^3, walls and the aligned layout's
    # i = N column included
    pos = sorted({0, 1, N // 2, N - 1, N})
    shapes = [_column_owner_cells(N, rows) for rows in (1, 2, 8)]
    shapes += [_kmarch_owner_cells(N, e, bx, kc) for e, bx, kc in ((4, 32, 1), (4, 128, 16), (2, 64, 4))]
    for n_shape, (i0, j, k, extra, V) in enumerate(shapes):
        for sj in pos:
            for sk in (0, N // 2, N):
                at = (j == sj) & (k == sk)
                a0, ex = i0[at], extra[at]
                for si in pos:
                    owners = np.sum(((si >= a0) & (si < a0 + V)) | (ex & (si == a0 + V)))
                    assert owners == 1, (n_shape, si, sj, sk)


@pytest.mark.parametrize("nx,ny,nz", [(130, 17, 1), (37, 29, 1), (5, 1, 1), (257, 66, 1), (33, 21, 5),
                                      (67, 13, 4), (45, 10, 8), (3, 2, 2), (512, 16, 8), (9, 3, 1)])
@pytest.mark.parametrize("esize", [4, 2])
@pytest.mark.parametrize("rows", [1, 2, 3, 8])
def test_scol_kernel_addresses(nx, ny, nz, esize, rows):
    # heat_scol_kernel (COLUMN_SMEM): thread (lane, ty) loads its own row of
    # every plane; rows y-1 and y+1 come from a shared slab of BY + 2 rows
    # (row 0 and BY + 1 are the block's halo rows, loaded by the first and
    # last thread rows).  With one thread row per block the same thread
    # loads both halo rows, each under its own condition.
    V = VEC[esize]
    is3d = nz > 1
    nzm = 8 if is3d else 1
    BY = max(1, min(rows, 8))
    grid = (-(-nx // (32 * V)), -(-ny // BY), 1)
    pitch = pitch_of(nx, esize)
    plane = pitch * ny
    size = plane * nz
    slabf = 32 * V
    smem = (BY + 2) * nzm * slabf  # floats (heat_scol_smem)
    bx, by, bz, lane, ty, _ = threads(grid, (32, BY, 1))
    x0 = (bx * 32 + lane) * V
    y0 = by * BY
    y = y0 + ty
    xin = x0 < nx
    act = xin & (y < ny)
    row_ld = np.minimum(y, ny - 1)
    written = set()
    covered = np.zeros(size, dtype=np.int64)
    blk = (bx * 65536 + by)
    for z in range(min(nz, nzm)):
        q = z * plane + row_ld * pitch + x0
        check_vec(q[act], V, (z * plane + row_ld * pitch)[act], pitch, size)
        m = act & (lane == 0) & (x0 > 0)
        check_vec((q - 1)[m], 1, (z * plane + row_ld * pitch)[m], pitch, size)
        m = act & (lane == 31) & (x0 + V < nx)
        check_vec((q + V)[m], 1, (z * plane + row_ld * pitch)[m], pitch, size)
        for side in (0, 1):
            want = ((ty == 0) & (y0 > 0)) if side == 0 else ((ty == BY - 1) & (y0 + BY < ny))
            m = xin & want
            hy = y0 - 1 if side == 0 else y0 + BY
            hr = 0 if side == 0 else BY + 1
            check_vec((z * plane + hy * pitch + x0)[m], V, (z * plane + hy * pitch)[m], pitch, size)
            off = (hr * nzm + z) * slabf + lane * V
            assert np.all(off[m] + V <= smem)
            written.update(zip(blk[m].tolist(), (off[m]).tolist()))
        off = ((ty + 1) * nzm + z) * slabf + lane * V
        assert np.all(off[act] + V <= smem)
        written.update(zip(blk[act].tolist(), off[act].tolist()))
    for z in range(min(nz, nzm)):  # after the barrier: rows y-1 and y+1 from the slab
        for cond, r in ((act & (y > 0), ty), (act & (y + 1 < ny), ty + 2)):
            off = (r * nzm + z) * slabf + lane * V
            for key in zip(blk[cond].tolist(), off[cond].tolist()):
                assert key in written, key
        nv = np.minimum(V, nx - x0)
        s0 = z * plane + y * pitch + x0
        check_vec(s0[act], nv[act], (z * plane + y * pitch)[act], pitch, size)
        for c in range(V):
            mm = act & (c < nv)
            np.add.at(covered, s0[mm] + c, 1)
    check_vec((y * pitch + x0)[act], V, (y * pitch)[act], pitch, ny * pitch)  # the P row
    cells = np.zeros((nz, ny, pitch), dtype=bool)
    cells[:, :, :nx] = True
    assert np.array_equal(covered.reshape(nz, ny, pitch) == 1, cells)


def _fused_march_owned_exactly(N, rows, kmarch, extra_in_every_block=False):
    """Whether the fused march's stores cover every element of the written
    set exactly once (f32); `extra_in_every_block` plants the mistake of
    giving every block's lane 31 the aligned layout's extra i = N cell."""
    V, esize = 4, 4
    M = Mk = N + 1
    aln = N % (32 * V) == 0
    pitch = pitch_of(M, esize)
    plane = pitch * M
    by_ = max(1, min(rows, 8))
    span = N if aln else M
    grid = (-(-span // (32 * V)), -(-M // by_), -(-Mk // kmarch))
    bx, by, bz, lane, ty, _ = threads(grid, (32, by_, 1))
    i0 = (bx * 32 + lane) * V
    j = by * by_ + ty
    k0 = bz * kmarch
    k1 = np.minimum(k0 + kmarch, Mk)
    act_i = np.ones_like(i0, dtype=bool) if aln else (i0 < M)
    owned = np.zeros(plane * Mk, dtype=np.int64)
    for p in range(min(kmarch, Mk)):
        k = k0 + p
        m = (j < M) & (k < k1) & act_i
        o = k * plane + j * pitch + i0
        nv = np.minimum(V, M - i0)
        for c in range(V):
            mc = m & (c < nv)
            np.add.at(owned, o[mc] + c, 1)
        if aln:
            mx = m & (lane == 31) & (extra_in_every_block | (i0 + V == N))
            np.add.at(owned, o[mx] + V, 1)
    cells = np.zeros((Mk, M, pitch), dtype=bool)
    cells[:, :, :M] = True
    return np.array_equal(owned.reshape(Mk, M, pitch) == 1, cells)


def test_planted_seam_mistake_fails_the_coverage_check():
    # the re-trace tells the aligned layout's extra cell apart: owned by the
    # last block's lane 31 the stores cover each element once; owned by
    # every block's lane 31 (two blocks along i at N = 256) the first
    # column of the second block is written twice
    assert _fused_march_owned_exactly(256, 4, 64)
    assert not _fused_march_owned_exactly(256, 4, 64, extra_in_every_block=True)
    # with one block along i (N = 128) the two rules agree
    assert _fused_march_owned_exactly(128, 4, 64, extra_in_every_block=True)
