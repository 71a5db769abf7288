"""Device-side batch loop (gs_plan.graph_loop = 1): one launch of a graph
whose conditional while node repeats the batch on the device must give the
same bits as per-step launches and as the unrolled batch graphs, for every
stencil, odd and even batch sizes (odd ones flip the buffer parity, so the
loop body holds two batches), changing trip counts on a cached loop graph,
and the explicit build/launch calls."""
import numpy as np
import pytest

import gs_inputs
from gsutil import (HEAT_RTOL, fdtd_concat, fdtd_read, fdtd_setup, fdtd_upload, heat_gpu, heat_read, heat_setup,
                    heat_upload, max_rel)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


@pytest.mark.parametrize("shape", [(97, 41, 1), (33, 21, 5), (130, 9, 17)])
def test_loop_bit_identical_to_per_step(shape):
    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=40)
    n = 37
    base = heat_gpu(T0, P, n, S=0)
    for S in (1, 2, 3, 7, 10, 18, 37, 50):
        got = heat_gpu(T0, P, n, S=S, plan=dict(graph_loop=1))
        assert np.array_equal(got, base), f"S={S}"
    # depth 2 resolves to COLUMN (2D, thin stacks) or STREAM (17 planes)
    for plan in (dict(graph_loop=1, use_pdl=1), dict(graph_loop=1, temporal_depth=2),
                 dict(graph_loop=1, temporal_depth=4)):
        for S in (5, 6):
            assert np.array_equal(heat_gpu(T0, P, n, S=S, plan=plan), base), f"S={S} {plan}"


def test_trip_count_changes_on_a_cached_loop_graph():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(70, 50, 1, seed=41)
    ctx, fields = heat_setup(70, 50, plan=dict(graph_loop=1))
    try:
        heat_upload(ctx, T0, P)
        for n in (23, 41, 8, 4, 16):  # trips 5, 10, 2, 1, 4 of the S=4 loop graph
            g.gs_step(ctx, n, 4)
        st = g.gs_get_stats(ctx)
        # one loop launch per call, plus one remainder graph for 23 and 41
        assert st["graph_launches"] == 5 + 2
        assert st["iterations"] == 92
        assert np.array_equal(heat_read(ctx, T0.shape), heat_gpu(T0, P, 92, S=0))
    finally:
        g.gs_destroy(ctx)
        del fields


def test_odd_batch_loop_bookkeeping():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(45, 38, 1, seed=42)
    ctx, fields = heat_setup(45, 38, plan=dict(graph_loop=1))
    try:
        heat_upload(ctx, T0, P)
        # S = 3 flips the parity: the body is two batches (2 trips), the
        # fifth batch runs as a plain batch graph, then the remainder of 2
        g.gs_step(ctx, 17, 3)
        st = g.gs_get_stats(ctx)
        assert st["graph_launches"] == 3
        assert g.gs_get_parity(ctx) == 1
        assert np.array_equal(heat_read(ctx, T0.shape), heat_gpu(T0, P, 17, S=0))
        # explicit build + launch: 6 batches of 3 -> one loop launch of 3 trips
        g.gs_graph_build(ctx, 3)
        assert g.gs_get_stats(ctx)["last_build_nodes"] == 6
        g.gs_graph_launch(ctx, 6)
        assert g.gs_get_parity(ctx) == 1  # 18 more steps keep it
        assert np.array_equal(heat_read(ctx, T0.shape), heat_gpu(T0, P, 35, S=0))
    finally:
        g.gs_destroy(ctx)
        del fields


def test_loop_plan_validation():
    import paper_2501_09398_gb300 as g

    ctx, fields = heat_setup(16, 8)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, graph_loop=2)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        # a device-launch graph may hold kernel, copy, set and child-graph nodes only
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, graph_loop=1, device_launch=1)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
        g.gs_set_plan(ctx, graph_loop=1)
        assert g.gs_get_plan(ctx)["graph_loop"] == 1
    finally:
        g.gs_destroy(ctx)
        del fields


def test_fdtd_loop_bit_identical():
    import paper_2501_09398_gb300 as g

    N, n = 20, 23
    out = []
    for S, plan in ((0, None), (5, dict(graph_loop=1)), (4, dict(graph_loop=1, use_pdl=1))):
        ctx, fields = fdtd_setup(N, plan=plan, src=(10, 10, 10))
        try:
            fdtd_upload(ctx, N, {})
            g.gs_step(ctx, n, S)
            out.append(fdtd_concat(fdtd_read(ctx, N)))
            assert g.gs_get_time(ctx) == n
        finally:
            g.gs_destroy(ctx)
            del fields
    assert np.any(out[0] != 0)
    assert np.array_equal(out[1], out[0]) and np.array_equal(out[2], out[0])


def test_skeleton_loop(oracle):
    import torch

    import paper_2501_09398_gb300 as g

    n = 10_000
    x0 = np.linspace(-2.0, 2.0, n).astype(np.float32)
    ctx = g.gs_create(g.GS_SKELETON, n, 1, 1, g.GS_F32, g.GS_BC_CLAMP, torch.cuda.current_stream().cuda_stream)
    buf = torch.from_numpy(x0).cuda()
    torch.cuda.synchronize()
    try:
        g.gs_bind_field(ctx, g.GS_FIELD_X, buf.data_ptr(), n)
        g.gs_set_scale(ctx, -1.0)
        g.gs_set_plan(ctx, graph_loop=1)
        g.gs_step(ctx, 1001, 100)  # 10 trips + a remainder of 1: odd count flips the sign
        g.gs_sync(ctx)
        assert np.array_equal(buf.cpu().numpy(), oracle.skeleton_run(x0, -1.0, 1001).astype(np.float32))
    finally:
        g.gs_destroy(ctx)


def test_config0_loop_full_size(oracle):
    # 2D 512x512, 1000 iterations as one device loop of 10 trips of 100
    T0, P = gs_inputs.heat_fields(512, 512, 1, seed=0)
    got = heat_gpu(T0, P, 1000, S=100, plan=dict(graph_loop=1))
    assert max_rel(got, oracle.heat_run(T0, P, 1000, oracle.HEAT_COEFFS_2D)) <= HEAT_RTOL
    assert np.array_equal(got, heat_gpu(T0, P, 1000, S=100))
