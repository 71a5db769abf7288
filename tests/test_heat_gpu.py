"""GPU parity of the thermal stencils against the FP64 oracle, through the C
ABI, plus bit-identity of every launch variant (per-step, graph-batched for
several S with remainder peeling, PDL edges, device-launch graphs, temporal
depth 2/4) and resume.

FP32 tolerance: max relative error <= 1e-5 (the bound stated for 1000
steps; short runs sit far below it)."""
import numpy as np
import pytest

import gs_inputs
from gsutil import HEAT_RTOL, heat_gpu, heat_read, heat_setup, heat_upload, max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401  (fails loudly if the library is missing)


def _coeffs(nz):
    import oracle

    return oracle.HEAT_COEFFS_2D if nz == 1 else oracle.HEAT_COEFFS_3D


# shapes span several blocks and ragged tails in x (vector width 4 or 8 and
# 32-lane warps), y (rows per block) and z (planes per block)
SHAPES_2D = [(130, 17), (37, 29), (5, 1), (1, 9), (4, 4), (257, 66), (1, 1)]
SHAPES_3D = [(33, 21, 5), (19, 7, 3), (130, 9, 17), (8, 8, 1), (3, 2, 2),
             (67, 13, 4), (45, 10, 8), (140, 6, 2),  # compile-time plane counts of the column kernel
             (70, 11, 24), (36, 9, 19)]  # the column kernel in 8-plane chunks


@pytest.mark.parametrize("shape", SHAPES_2D)
@pytest.mark.parametrize("bc", [0, 1])
def test_heat2d_parity_small(oracle, shape, bc):
    nx, ny = shape
    T0, P = gs_inputs.heat_fields(nx, ny, 1, seed=7)
    ref = oracle.heat_run(T0, P, 60, oracle.HEAT_COEFFS_2D, bc)
    for plan in (None, dict(block_x=32, rows=3)):
        got = heat_gpu(T0, P, 60, S=0, bc=bc, plan=plan)
        if bc == 1:  # Dirichlet drives values toward 0 at the edge: compare absolutely
            assert np.max(np.abs(got - ref)) <= HEAT_RTOL * np.max(np.abs(ref))
        else:
            assert max_rel(got, ref) <= HEAT_RTOL


@pytest.mark.parametrize("shape", SHAPES_3D)
@pytest.mark.parametrize("bc", [0, 1])
def test_heat3d_parity_small(oracle, shape, bc):
    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=8)
    ref = oracle.heat_run(T0, P, 40, oracle.HEAT_COEFFS_3D, bc)
    import paper_2501_09398_gb300 as g

    plans = [None, dict(block_x=64, rows=2), dict(kernel=g.GS_KERNEL_COLUMN, rows=3)]
    for plan in plans:
        got = heat_gpu(T0, P, 40, S=0, bc=bc, plan=plan)
        assert np.max(np.abs(got - ref)) <= HEAT_RTOL * np.max(np.abs(ref))


def test_heat3d_with_one_layer_equals_2d():
    # cz2*(U+D-2T) vanishes exactly when both neighbours clamp to the cell.
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(70, 33, 1, seed=9)
    a = heat_gpu(T0, P, 25, kind=g.GS_HEAT2D)
    b = heat_gpu(T0[None], P, 25, kind=g.GS_HEAT3D)[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("nz", [1, 4])
def test_graph_batches_bit_identical_to_per_step(nz):
    T0, P = gs_inputs.heat_fields(97, 41, nz, seed=10)
    n = 37
    base = heat_gpu(T0, P, n, S=0)
    for S in (1, 2, 3, 7, 10, 37, 50):
        assert np.array_equal(heat_gpu(T0, P, n, S=S), base), f"S={S}"
    for plan in (dict(use_pdl=1), dict(device_launch=1)):
        for S in (0, 5, 8):
            assert np.array_equal(heat_gpu(T0, P, n, S=S, plan=plan), base), f"S={S} {plan}"


def test_remainder_graphs_of_one_size_are_kept():
    """gs_step keeps the peeled remainder graphs of the latest remainder size
    only: returning to an earlier remainder builds its graph again, and the
    results stay bit-identical to per-step launches."""
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(97, 41, 1, seed=11)
    calls = (37, 38, 37, 37)  # remainders 7, 8, 7, 7 of S = 10
    base = heat_gpu(T0, P, sum(calls), S=0)
    ctx, fields = heat_setup(97, 41)
    try:
        heat_upload(ctx, T0, P)
        built = []
        for n in calls:
            g.gs_step(ctx, n, 10)
            built.append(g.gs_get_stats(ctx)["graphs_built"])
        got = heat_read(ctx, T0.shape)
    finally:
        g.gs_destroy(ctx)
        del fields
    assert np.array_equal(got, base)
    # call 3 rebuilt a remainder graph of 7 (call 2 dropped the ones of 7);
    # call 4 adds at most the remainder of 7 at the other buffer parity
    assert built[2] > built[1]
    assert built[3] - built[2] <= 1


@pytest.mark.parametrize("shape", [(96, 64, 1), (77, 45, 1), (300, 37, 1), (40, 33, 8), (21, 19, 3), (250, 20, 16),
                                   (500, 130, 1), (3, 2, 1), (40, 33, 4), (130, 9, 5), (64, 70, 2), (29, 3, 8),
                                   (40, 33, 12), (29, 3, 13), (130, 9, 9)])
@pytest.mark.parametrize("depth", [1, 2, 4])
def test_temporal_blocking_bit_identical(shape, depth):
    import paper_2501_09398_gb300 as g

    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=12)
    n = 4 * depth + 3  # peels n % depth single steps
    base = heat_gpu(T0, P, n, S=0, plan=dict(kernel=g.GS_KERNEL_MARCH, block_x=32, rows=5))
    # wavefront kernel: warps march `rows` rows; 2D stacks block_x/32 warps
    for rows, bx in ((16, 32), (3, 128), (1, 64)):
        plan = dict(temporal_depth=depth, kernel=g.GS_KERNEL_WAVE, rows=rows, block_x=bx)
        assert np.array_equal(heat_gpu(T0, P, n, S=0, plan=plan), base), f"wave rows={rows} bx={bx}"
        assert np.array_equal(heat_gpu(T0, P, n, S=6, plan=plan), base), f"wave graph rows={rows} bx={bx}"
    if depth == 1:  # column kernels: every plane of a column (of an 8-plane chunk when nz > 8) in registers
        for rows, kern in ((1, g.GS_KERNEL_COLUMN), (4, g.GS_KERNEL_COLUMN), (8, g.GS_KERNEL_COLUMN),
                           (1, g.GS_KERNEL_COLUMN_SMEM), (3, g.GS_KERNEL_COLUMN_SMEM), (8, g.GS_KERNEL_COLUMN_SMEM)):
            plan = dict(kernel=kern, rows=rows)
            if nz > 8 and kern == g.GS_KERNEL_COLUMN_SMEM:
                with pytest.raises(g.GsError):
                    heat_gpu(T0, P, n, S=0, plan=plan)
                continue
            assert np.array_equal(heat_gpu(T0, P, n, S=0, plan=plan), base), f"column {kern} rows={rows}"
            assert np.array_equal(heat_gpu(T0, P, n, S=5, plan=plan), base), f"column {kern} graph rows={rows}"
    if depth > 1:  # column kernel at depth 2 / 4: levels in registers (2D, stacks of <= 8 planes, and at
        # depth 2 deeper stacks marched in z chunks of tile_y planes)
        for bx, rows, chunk in ((32, 0, 1), (64, 2, 5), (128, 0, 3), (256, 0, 0)):
            plan = dict(temporal_depth=depth, kernel=g.GS_KERNEL_COLUMN, block_x=bx, rows=rows, tile_y=chunk)
            if nz > 8 and depth == 4:
                with pytest.raises(g.GsError):
                    heat_gpu(T0, P, n, S=0, plan=plan)
                continue
            assert np.array_equal(heat_gpu(T0, P, n, S=0, plan=plan), base), f"column depth={depth} bx={bx}"
            assert np.array_equal(heat_gpu(T0, P, n, S=5, plan=plan), base), f"column graph depth={depth} bx={bx}"
            assert np.array_equal(heat_gpu(T0, P, n, S=0, bc=1, plan=plan), heat_gpu(T0, P, n, S=0, bc=1)), \
                f"column dirichlet depth={depth} bx={bx}"
    if depth > 1:  # overlapped shared-memory tiles
        for tile in ((32, 32), (16, 8), (13, 7)):
            plan = dict(temporal_depth=depth, kernel=g.GS_KERNEL_TILE, tile_x=tile[0], tile_y=tile[1])
            assert np.array_equal(heat_gpu(T0, P, n, S=0, plan=plan), base), f"tile={tile}"
            assert np.array_equal(heat_gpu(T0, P, n, S=6, plan=plan), base), f"tile graph={tile}"
    b1 = heat_gpu(T0, P, n, S=0, bc=1)
    assert np.array_equal(heat_gpu(T0, P, n, S=0, bc=1, plan=dict(temporal_depth=depth, kernel=g.GS_KERNEL_WAVE)),
                          b1)


def test_wave_kernel_rejects_deep_stacks():
    import paper_2501_09398_gb300 as g

    ctx, fields = heat_setup(40, 20, 17)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, temporal_depth=2, kernel=g.GS_KERNEL_WAVE)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
        g.gs_set_plan(ctx, temporal_depth=2)  # AUTO streams the planes through shared memory at depth 2
        assert g.gs_get_plan(ctx)["kernel"] == g.GS_KERNEL_STREAM
        g.gs_set_plan(ctx, temporal_depth=2, block_x=128)  # and marches in registers with another block shape
        assert g.gs_get_plan(ctx)["kernel"] == g.GS_KERNEL_COLUMN
        g.gs_set_plan(ctx, temporal_depth=4)  # and the tile kernel at depth 4
        assert g.gs_get_plan(ctx)["kernel"] == g.GS_KERNEL_TILE
    finally:
        g.gs_destroy(ctx)
        del fields


def test_resume_is_bit_identical():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(64, 48, 1, seed=13)
    full = heat_gpu(T0, P, 30, S=4)
    ctx, fields = heat_setup(64, 48)
    try:
        heat_upload(ctx, T0, P)
        g.gs_step(ctx, 11, 4)
        mid = heat_read(ctx, T0.shape)
        heat_upload(ctx, mid, P)  # checkpoint round trip through the host
        g.gs_step(ctx, 19, 4)
        assert np.array_equal(heat_read(ctx, T0.shape), full)
        st = g.gs_get_stats(ctx)
        assert st["iterations"] == 30
    finally:
        g.gs_destroy(ctx)


def test_config0_full_size(oracle):
    # 2D 512x512, 1000 iterations, graph batches of 100 and per-step launch
    T0, P = gs_inputs.heat_fields(512, 512, 1, seed=0)
    ref = oracle.heat_run(T0, P, 1000, oracle.HEAT_COEFFS_2D)
    got = heat_gpu(T0, P, 1000, S=100)
    err = max_rel(got, ref)
    print(f"config0 max rel err {err:.3e}")
    assert err <= HEAT_RTOL
    assert np.array_equal(heat_gpu(T0, P, 1000, S=0), got)
    # the column kernel at temporal depth 2 and 4 (AUTO in 2D)
    for depth in (2, 4):
        assert np.array_equal(heat_gpu(T0, P, 1000, S=100, plan=dict(temporal_depth=depth, block_x=256)), got)


def test_config1_full_size(oracle):
    # 3D 512x512x8, 1000 iterations, temporal depth 1/2/4 bit-identical
    T0, P = gs_inputs.heat_fields(512, 512, 8, seed=0)
    ref = oracle.heat_run(T0, P, 1000, oracle.HEAT_COEFFS_3D)
    got = heat_gpu(T0, P, 1000, S=100)
    err = max_rel(got, ref)
    print(f"config1 max rel err {err:.3e}")
    assert err <= HEAT_RTOL
    for depth in (2, 4):
        assert np.array_equal(heat_gpu(T0, P, 1000, S=100, plan=dict(temporal_depth=depth)), got)


def test_deep_stack_full_size(oracle):
    # 256^3: the column kernel in 8-plane chunks (the default above 8 planes)
    # against the oracle, and bit for bit against the MARCH kernel
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(256, 256, 256, seed=0)
    n = 12
    got = heat_gpu(T0, P, n, S=5)
    ref = oracle.heat_run(T0, P, n, oracle.HEAT_COEFFS_3D)
    assert max_rel(got, ref) <= HEAT_RTOL
    march = heat_gpu(T0, P, n, S=0, plan=dict(kernel=g.GS_KERNEL_MARCH, block_x=64, rows=8))
    assert np.array_equal(march, got)
    # depth 2 marched in z (chunks of 32 planes; 13 steps: 6 fused launches and one single step)
    zm = heat_gpu(T0, P, n, S=5, plan=dict(kernel=g.GS_KERNEL_COLUMN, temporal_depth=2, block_x=128))
    assert np.array_equal(zm, got)


def test_large_2d_sampled(oracle):
    # 4096^2 at the bench's launch shape: the oracle checks a 40-step run on
    # a 160x160 window whose dependence cone (radius 40) stays inside it.
    T0, P = gs_inputs.heat_fields(4096, 4096, 1, seed=0)
    got = heat_gpu(T0, P, 40, S=20)
    y0, x0, w, n = 2000, 3900, 160, 40
    sub = oracle.heat_run(T0[y0:y0 + w, x0:x0 + w], P[y0:y0 + w, x0:x0 + w], n, oracle.HEAT_COEFFS_2D)
    inner = slice(n, w - n)
    assert max_rel(got[y0:y0 + w, x0:x0 + w][inner, inner], sub[inner, inner]) <= HEAT_RTOL
    # and the grid's own corner, where the clamp boundary is inside the window
    sub = oracle.heat_run(T0[-w:, -w:], P[-w:, -w:], n, oracle.HEAT_COEFFS_2D)
    assert max_rel(got[-w + n:, -w + n:], sub[n:, n:]) <= HEAT_RTOL
    # the bench's temporally blocked plan (column kernel, depth 2) gives the same bits
    assert np.array_equal(heat_gpu(T0, P, 40, S=20, plan=dict(temporal_depth=2, block_x=64)), got)


def test_zero_iterations_and_state_errors():
    import paper_2501_09398_gb300 as g

    ctx = g.gs_create(g.GS_HEAT2D, 16, 8, 1, g.GS_F32, g.GS_BC_CLAMP, None)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_step(ctx, 5, 0)
        assert e.value.status == g.GS_ERR_STATE
        fields = g.HeatFields(ctx, 16, 8)
        g.gs_step(ctx, 0, 7)  # no-op
        assert g.gs_get_parity(ctx) == 0
        with pytest.raises(g.GsError) as e:
            g.gs_step(ctx, -1, 0)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        with pytest.raises(g.GsError) as e:
            g.gs_graph_launch(ctx, 1)
        assert e.value.status == g.GS_ERR_STATE
        with pytest.raises(g.GsError) as e:
            g.gs_bind_field(ctx, g.GS_FIELD_T0, fields.T0.data_ptr() + 4, fields.pitch)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        with pytest.raises(g.GsError) as e:
            g.gs_bind_field(ctx, g.GS_FIELD_T0, fields.T0.data_ptr(), 18)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, temporal_depth=3)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, use_pdl=1, device_launch=1)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        with pytest.raises(g.GsError) as e:
            g.gs_upload(ctx, g.GS_FIELD_T, np.zeros(5, dtype=np.float32))
        assert e.value.status == g.GS_ERR_INVALID_ARG
        with pytest.raises(g.GsError) as e:
            g.gs_set_heat_coeffs(ctx, k=float("nan"))
        assert e.value.status == g.GS_ERR_NUMERIC
        # odd S flips parity per launch; the state follows
        T0, P = gs_inputs.heat_fields(16, 8, 1, seed=1)
        heat_upload(ctx, T0, P)
        g.gs_graph_build(ctx, 3)
        g.gs_graph_launch(ctx, 3)
        assert g.gs_get_parity(ctx) == 1
        st = g.gs_get_stats(ctx)
        assert st["last_build_nodes"] == 3 and st["last_build_seconds"] > 0
        assert np.array_equal(heat_read(ctx, T0.shape), heat_gpu(T0, P, 9, S=0))
        del fields
    finally:
        g.gs_destroy(ctx)
