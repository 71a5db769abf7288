"""Block traversal order (gs_plan.traverse): walking every other launch's
blocks last to first keeps the rows the previous step touched last in L2;
the order never changes a result.  Checked bit for bit for every thermal
kernel variant (2D and 3D, both boundaries, per-step and graph batches with
an odd batch size), the FDTD half-steps (vacuum and media) and the fused
multi-instance batch; invalid values are rejected."""
import numpy as np
import pytest

import gs_inputs
from gsutil import FDTD_NAMES, fdtd_read, fdtd_setup, fdtd_upload, heat_gpu, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _plans(g, nz):
    out = [dict(kernel=g.GS_KERNEL_MARCH, block_x=32, rows=5),
           dict(kernel=g.GS_KERNEL_WAVE, temporal_depth=2, rows=3, block_x=64),
           dict(kernel=g.GS_KERNEL_TILE, temporal_depth=4, tile_x=16, tile_y=8)]
    if nz <= 8:
        out += [dict(kernel=g.GS_KERNEL_COLUMN, rows=4), dict(kernel=g.GS_KERNEL_COLUMN_SMEM, rows=3)]
    if nz > 1:
        out += [dict(kernel=g.GS_KERNEL_COLUMN, temporal_depth=2, block_x=64),
                dict(kernel=g.GS_KERNEL_STREAM, temporal_depth=2, block_x=256, tile_y=3)]
    return out


@pytest.mark.parametrize("shape", [(300, 37, 1), (130, 45, 8), (77, 20, 3)])
@pytest.mark.parametrize("bc", [0, 1])
def test_heat_traversal_order_bit_identical(shape, bc):
    import paper_2501_09398_gb300 as g

    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=21)
    n = 11
    for plan in _plans(g, nz):
        fwd = heat_gpu(T0, P, n, S=0, bc=bc, plan=dict(plan, traverse=g.GS_TRAVERSE_FORWARD))
        for S in (0, 5):
            alt = heat_gpu(T0, P, n, S=S, bc=bc, plan=dict(plan, traverse=g.GS_TRAVERSE_ALTERNATE))
            assert np.array_equal(alt, fwd), f"{plan} S={S}"


@pytest.mark.parametrize("media", [False, True])
def test_fdtd_traversal_order_bit_identical(media):
    import paper_2501_09398_gb300 as g

    N, n = 37, 9
    init = gs_inputs.fdtd_random_all(N, seed=22)
    med = gs_inputs.fdtd_media(N, n_mat=4, seed=23) if media else None
    res = []
    for tr in (g.GS_TRAVERSE_FORWARD, g.GS_TRAVERSE_ALTERNATE):
        for plan in (dict(rows=2), dict(kernel=g.GS_KERNEL_MARCH, block_x=64, rows=4),
                     dict(kernel=g.GS_KERNEL_FUSED, rows=2), dict(kernel=g.GS_KERNEL_FUSED, rows=4, tile_y=5)):
            if media and (plan.get("kernel") == g.GS_KERNEL_MARCH or plan == dict(kernel=g.GS_KERNEL_FUSED, rows=2)):
                continue
            ctx, fields = fdtd_setup(N, plan=dict(plan, traverse=tr), src=(10, 20, 30), media=med)
            try:
                fdtd_upload(ctx, N, init)
                g.gs_step(ctx, n, 4)
                res.append(fdtd_read(ctx, N))
            finally:
                g.gs_destroy(ctx)
                del fields
    for r in res[1:]:
        assert all(np.array_equal(r[k], res[0][k]) for k in FDTD_NAMES)


def test_multi_traversal_order_bit_identical():
    import paper_2501_09398_gb300 as g

    sides = [70, 300, 129, 64, 257]
    inputs = gs_inputs.instance_fields(sides, seed_base=40)
    out = []
    for tr in (g.GS_TRAVERSE_FORWARD, g.GS_TRAVERSE_ALTERNATE):
        for kernel in (g.GS_KERNEL_MARCH, g.GS_KERNEL_COLUMN):
            m = g.gs_multi_create(sides, sides, g.GS_F32, g.GS_BC_CLAMP, stream_handle())
            fields = g.MultiFields(m, sides, sides)
            try:
                g.gs_multi_set_plan(m, kernel=kernel, traverse=tr)
                for i, (T, P) in enumerate(inputs):
                    g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
                    g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
                g.gs_multi_step(m, 13, 5, g.GS_MULTI_FUSED)
                out.append([g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T))
                            for i, (T, _) in enumerate(inputs)])
            finally:
                g.gs_multi_destroy(m)
                del fields
    for o in out[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(o, out[0]))


def test_invalid_traverse_rejected():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(40, 30, 1, seed=24)
    with pytest.raises(g.GsError):
        heat_gpu(T0, P, 1, plan=dict(traverse=3))
