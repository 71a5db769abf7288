"""Slab decomposition on one GPU: a grid split into 2-4 sub-domains with halo
copies between every launch must give the undivided grid's result bit for
bit (2D thermal 512^2, 3D thermal 512x512x8, FDTD 64^3 with the source, and
ragged splits), per-step and in batch graphs with a peeled remainder, with
and without PDL, at temporal depths the halo allows (a deep stack also with
the STREAM kernel at depth 2)."""
import numpy as np
import pytest

import gs_inputs
from gsutil import heat_gpu, fdtd_concat, fdtd_read, fdtd_setup, fdtd_upload, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def slab_heat(T0, P, n, S, K, halo=1, plan=None, dtype="f32", bc=0):
    import paper_2501_09398_gb300 as g

    nz = 1 if T0.ndim == 2 else T0.shape[0]
    ny, nx = T0.shape[-2:]
    kind = g.GS_HEAT2D if nz == 1 else g.GS_HEAT3D
    s = g.gs_slab_create(kind, nx, ny, nz, K, halo, g.DTYPES[dtype], bc, stream_handle())
    try:
        if plan:
            g.gs_slab_set_plan(s, **plan)
        g.gs_slab_upload(s, g.GS_FIELD_T, np.ascontiguousarray(T0, dtype=np.float32))
        g.gs_slab_upload(s, g.GS_FIELD_P, np.ascontiguousarray(P, dtype=np.float32))
        g.gs_slab_step(s, n, S)
        out = g.gs_slab_read_field(s, g.GS_FIELD_T, np.empty(T0.shape, dtype=np.float32))
        ext = [g.gs_slab_extent(s, k) for k in range(K)]
        stats = g.gs_slab_get_stats(s)
    finally:
        g.gs_slab_destroy(s)
    return out, ext, stats


def test_partition_covers_the_axis():
    T0, P = gs_inputs.heat_fields(97, 41, 1, seed=1)
    _, ext, _ = slab_heat(T0, P, 1, 0, 3)
    assert ext == [(0, 14), (14, 14), (28, 13)]


@pytest.mark.parametrize("K", [2, 4])
def test_config0_slabs_bit_identical(K):
    # 2D 512^2 (configuration 0's grid), split along y
    T0, P = gs_inputs.heat_fields(512, 512, 1, seed=0)
    n = 137
    base = heat_gpu(T0, P, n, S=0)
    for S in (0, 10, 100):  # per-step; 13 batches + a remainder of 7; one batch + 37
        got, _, st = slab_heat(T0, P, n, S, K)
        assert np.array_equal(got, base), (K, S)
        if S:
            assert st["graphs_built"] >= 1 and st["last_build_nodes"] > 0
    got, _, _ = slab_heat(T0, P, n, 10, K, plan=dict(use_pdl=1))
    assert np.array_equal(got, base), "PDL"


@pytest.mark.parametrize("K", [2, 4])
@pytest.mark.parametrize("depth", [2, 4])
def test_config0_slabs_temporal_depth(K, depth):
    T0, P = gs_inputs.heat_fields(512, 512, 1, seed=0)
    n = 50  # depth 4: 12 fused launches and 2 single steps
    plan = dict(temporal_depth=depth, kernel=4, block_x=64)
    base = heat_gpu(T0, P, n, S=0, plan=plan)
    for S in (0, 16):
        got, _, _ = slab_heat(T0, P, n, S, K, halo=depth, plan=plan)
        assert np.array_equal(got, base), (K, depth, S)


@pytest.mark.parametrize("K", [2, 4])
def test_config1_slabs_bit_identical(K):
    # 3D 512x512x8 (configuration 1's grid), split along z
    T0, P = gs_inputs.heat_fields(512, 512, 8, seed=0)
    n = 61
    base = heat_gpu(T0, P, n, S=0)
    for S in (0, 20):
        got, _, _ = slab_heat(T0, P, n, S, K)
        assert np.array_equal(got, base), (K, S)
    got, _, _ = slab_heat(T0, P, n, 20, K, plan=dict(use_pdl=1))
    assert np.array_equal(got, base), "PDL"


def test_config1_slabs_wave_depth2():
    T0, P = gs_inputs.heat_fields(512, 512, 8, seed=0)
    plan = dict(temporal_depth=2, kernel=2, block_x=64, rows=4)
    base = heat_gpu(T0, P, 41, S=0, plan=plan)
    got, _, _ = slab_heat(T0, P, 41, 10, 4, halo=2, plan=plan)
    assert np.array_equal(got, base)


@pytest.mark.parametrize("shape,K,dtype,bc", [((97, 41, 1), 3, "f32", 0), ((97, 41, 1), 3, "bf16", 1),
                                              ((40, 33, 7), 3, "f32", 1), ((40, 33, 19), 2, "f16", 0),
                                              ((130, 9, 1), 4, "f32", 0)])
def test_ragged_slabs_bit_identical(shape, K, dtype, bc):
    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=3)
    n = 23
    base = heat_gpu(T0, P, n, S=0, dtype=dtype, bc=bc)
    for S in (0, 5):
        got, _, _ = slab_heat(T0, P, n, S, K, dtype=dtype, bc=bc)
        assert np.array_equal(got, base), (shape, K, S)


@pytest.mark.parametrize("K", [2, 3])
def test_deep_stack_slabs_stream_depth2(K):
    # a deep stack split along z, each slab stepped by the STREAM kernel at
    # depth 2 (planes streamed through shared memory), halo 2
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(130, 40, 37, seed=5)
    n = 23  # eleven depth-2 launches and one single step
    base = heat_gpu(T0, P, n, S=0)
    plan = dict(temporal_depth=2, kernel=g.GS_KERNEL_STREAM, block_x=256, tile_y=5)
    for S in (0, 6):
        got, _, _ = slab_heat(T0, P, n, S, K, halo=2, plan=plan)
        assert np.array_equal(got, base), (K, S)
    assert g.gs_wait_timeouts() == 0


def slab_fdtd(N, n, S, K, src, plan=None, dtype="f32"):
    import paper_2501_09398_gb300 as g

    s = g.gs_slab_create(g.GS_FDTD3D, N, N, N, K, 1, g.DTYPES[dtype], g.GS_BC_PEC, stream_handle())
    try:
        g.gs_slab_set_fdtd_params(s, courant=0.5, src_on=1, src=src)
        if plan:
            g.gs_slab_set_plan(s, **plan)
        z = np.zeros((N + 1,) * 3, dtype=np.float32)
        for fid in g.FDTD_FIELDS:
            g.gs_slab_upload(s, fid, z)
        g.gs_slab_step(s, n, S)
        out = {nm: g.gs_slab_read_field(s, fid, np.empty((N + 1,) * 3, dtype=np.float32))
               for fid, nm in zip(g.FDTD_FIELDS, ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"))}
    finally:
        g.gs_slab_destroy(s)
    return out


def fdtd_single(N, n, src, plan=None, dtype="f32"):
    import paper_2501_09398_gb300 as g

    ctx, fields = fdtd_setup(N, dtype=dtype, plan=plan, src=src)
    try:
        fdtd_upload(ctx, N, {})
        g.gs_step(ctx, n, 0)
        return fdtd_read(ctx, N)
    finally:
        g.gs_destroy(ctx)
        del fields


@pytest.mark.parametrize("K", [2, 4])
def test_fdtd64_slabs_bit_identical(K):
    N, n = 64, 90
    src = (32, 32, 32)
    base = fdtd_concat(fdtd_single(N, n, src))
    assert np.abs(base).max() > 0
    for S in (0, 7, 45):
        got = fdtd_concat(slab_fdtd(N, n, S, K, src))
        assert np.array_equal(got, base), (K, S)
    got = fdtd_concat(slab_fdtd(N, n, 7, K, src, plan=dict(use_pdl=1)))
    assert np.array_equal(got, base), "PDL"


@pytest.mark.parametrize("src", [(10, 20, 16), (33, 31, 17), (5, 5, 0), (7, 9, 64)])
def test_fdtd_slab_source_on_every_slab_boundary(src):
    # K = 4 over 65 planes: slabs own planes [0, 17), [17, 33), [33, 49), [49, 65);
    # sources on the first / last owned planes and the walls
    N, n = 64, 40
    base = fdtd_concat(fdtd_single(N, n, src))
    got = fdtd_concat(slab_fdtd(N, n, 9, 4, src))
    assert np.array_equal(got, base)


def test_fdtd_slab_march_kernel_and_bf16():
    N, n, src = 37, 30, (18, 18, 18)
    plan = dict(kernel=1, rows=4, block_x=32)
    base = fdtd_concat(fdtd_single(N, n, src, plan=plan))
    assert np.array_equal(fdtd_concat(slab_fdtd(N, n, 6, 3, src, plan=plan)), base)
    base = fdtd_concat(fdtd_single(N, n, src, dtype="bf16"))
    assert np.array_equal(fdtd_concat(slab_fdtd(N, n, 6, 3, src, dtype="bf16")), base)


def test_slab_refusals():
    import paper_2501_09398_gb300 as g

    h = stream_handle()
    with pytest.raises(g.GsError) as e:
        g.gs_slab_create(g.GS_HEAT2D, 64, 10, 1, 4, 3, g.GS_F32, g.GS_BC_CLAMP, h)  # 2 rows a slab < halo 3
    assert e.value.status == g.GS_ERR_INVALID_ARG
    s = g.gs_slab_create(g.GS_HEAT2D, 64, 64, 1, 2, 2, g.GS_F32, g.GS_BC_CLAMP, h)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_slab_set_plan(s, temporal_depth=4, kernel=4)
        assert e.value.status == g.GS_ERR_UNSUPPORTED and "halo" in str(e.value)
        with pytest.raises(g.GsError) as e:
            g.gs_slab_set_plan(s, graph_loop=1)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
        with pytest.raises(g.GsError) as e:
            g.gs_slab_upload(s, g.GS_FIELD_T, np.zeros((63, 64), dtype=np.float32))
        assert e.value.status == g.GS_ERR_INVALID_ARG
    finally:
        g.gs_slab_destroy(s)
