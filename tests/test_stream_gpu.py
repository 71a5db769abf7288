"""The STREAM kernel (3D thermal at temporal depth 2, planes streamed through
shared memory by tensor copies): bit-identical to the depth-1 COLUMN path,
which the oracle checks, on ragged shapes in every storage type under both
boundaries, with 8 and 16 compute warps, chunks of 1, 5 and 32 planes,
per-step and in graph batches with peeled remainders and PDL; at full size on
the 256^3 stack and the 512x512x8 configuration; no bounded wait runs out."""
import numpy as np
import pytest

import gs_inputs
from gsutil import heat_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def stream_plan(block_x=256, chunk=32, pdl=0):
    import paper_2501_09398_gb300 as g

    return dict(kernel=g.GS_KERNEL_STREAM, temporal_depth=2, block_x=block_x, tile_y=chunk, use_pdl=pdl)


@pytest.mark.parametrize("shape", [(97, 41, 9), (130, 30, 17), (256, 64, 40), (40, 33, 4), (29, 3, 13), (128, 28, 8),
                                   (5, 3, 33), (300, 15, 2), (128, 14, 3)])
@pytest.mark.parametrize("dtype,bc", [("f32", 0), ("f32", 1), ("bf16", 0), ("f16", 1)])
def test_stream_bit_identical_to_depth1(shape, dtype, bc):
    import paper_2501_09398_gb300 as g

    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=nx + ny + nz)
    n = 13  # six fused launches, then one single step
    base = heat_gpu(T0, P, n, S=0, dtype=dtype, bc=bc)
    for bx, chunk in ((256, 32), (512, 5), (256, 1)):
        got = heat_gpu(T0, P, n, S=0, dtype=dtype, bc=bc, plan=stream_plan(bx, chunk))
        assert np.array_equal(got, base), (bx, chunk)
    got = heat_gpu(T0, P, n, S=4, dtype=dtype, bc=bc, plan=stream_plan(256, 7))
    assert np.array_equal(got, base), "graph batches"
    got = heat_gpu(T0, P, n, S=5, dtype=dtype, bc=bc, plan=stream_plan(512, 32, pdl=1))
    assert np.array_equal(got, base), "PDL"
    assert g.gs_wait_timeouts() == 0


def test_stream_full_size_deep_stack():
    # 256^3: the bench's deep-stack workload, 12 steps in batches of 5
    T0, P = gs_inputs.heat_fields(256, 256, 256, seed=0)
    import paper_2501_09398_gb300 as g

    base = heat_gpu(T0, P, 12, S=5)
    for bx, chunk in ((256, 32), (512, 32), (256, 17)):
        assert np.array_equal(heat_gpu(T0, P, 12, S=5, plan=stream_plan(bx, chunk)), base), (bx, chunk)
    assert g.gs_wait_timeouts() == 0


def test_stream_full_size_thin_stack():
    # 512x512x8 (the bench's default grid), 1000 iterations in batches of 100
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(512, 512, 8, seed=0)
    base = heat_gpu(T0, P, 1000, S=100)
    for chunk in (8, 4):
        assert np.array_equal(heat_gpu(T0, P, 1000, S=100, plan=stream_plan(256, chunk)), base), chunk
    assert g.gs_wait_timeouts() == 0


@pytest.mark.parametrize("kind,nz,plan,status", [
    ("HEAT2D", 1, dict(temporal_depth=2), "INVALID_ARG"),
    ("HEAT3D", 8, dict(temporal_depth=1), "INVALID_ARG"),
    ("HEAT3D", 8, dict(temporal_depth=4), "INVALID_ARG"),
    ("HEAT3D", 8, dict(temporal_depth=2, block_x=128), "INVALID_ARG"),
    ("HEAT3D", 8, dict(temporal_depth=2, tile_y=-1), "INVALID_ARG"),
])
def test_stream_plan_refusals(kind, nz, plan, status):
    import paper_2501_09398_gb300 as g

    ctx = g.gs_create(getattr(g, "GS_" + kind), 64, 64, nz)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, kernel=g.GS_KERNEL_STREAM, **plan)
        assert e.value.status == getattr(g, "GS_ERR_" + status)
    finally:
        g.gs_destroy(ctx)
