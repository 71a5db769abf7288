"""Error paths under host-side fault injection: an allocation or a graph
kernel-node addition made to fail (gs_debug_inject_failure) returns its
status, leaks no device memory, launches nothing, and leaves the context,
instance batch or slab set usable, with results bit-identical to a run that
never failed.  No GPU fault is involved: the failures are returned
statuses."""
import numpy as np
import pytest

import gs_inputs
from gsutil import heat_gpu, heat_read, heat_setup, heat_upload, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


@pytest.fixture(autouse=True)
def _disarm():
    import paper_2501_09398_gb300 as g

    g.gs_debug_inject_failure(g.GS_INJECT_NONE)
    yield
    g.gs_debug_inject_failure(g.GS_INJECT_NONE)


def _free():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("S,n,after,plan", [(10, 37, 4, {}), (7, 37, 9, {}), (7, 37, 3, {}), (10, 37, 12, {}),
                                            (10, 40, 3, dict(graph_loop=1)), (7, 40, 8, dict(graph_loop=1))])
def test_failed_graph_build_changes_nothing(S, n, after, plan):
    # S = 7 flips the buffer parity: the batch graphs of both parities are
    # built first, then the remainder's; a failure at any node of any of
    # them must leave the state and the time untouched
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(97, 41, 1, seed=21)
    base = heat_gpu(T0, P, n, S=0)
    ctx, fields = heat_setup(97, 41, plan=plan or None)
    try:
        heat_upload(ctx, T0, P)
        built0 = g.gs_get_stats(ctx)["graphs_built"]
        g.gs_debug_inject_failure(g.GS_INJECT_GRAPH_NODE, after)
        with pytest.raises(g.GsError) as e:
            g.gs_step(ctx, n, S)
        assert e.value.status == g.GS_ERR_CUDA, str(e.value)
        assert not g.gs_debug_injection_pending()
        st = g.gs_get_stats(ctx)
        assert st["graph_launches"] == 0 and st["iterations"] == 0 and g.gs_get_time(ctx) == 0
        assert g.gs_get_parity(ctx) == 0
        assert np.array_equal(heat_read(ctx, T0.shape), T0.astype(np.float32))
        assert st["graphs_built"] >= built0
        g.gs_step(ctx, n, S)  # the same call now succeeds
        assert np.array_equal(heat_read(ctx, T0.shape), base)
    finally:
        g.gs_destroy(ctx)
        del fields


def test_failed_fdtd_create_and_allocations_leak_nothing():
    import paper_2501_09398_gb300 as g

    h = stream_handle()
    free0 = _free()
    for _ in range(3):
        g.gs_debug_inject_failure(g.GS_INJECT_MALLOC, 0)  # the step counter
        with pytest.raises(g.GsError) as e:
            g.gs_create(g.GS_FDTD3D, 16, 16, 16, g.GS_F32, g.GS_BC_PEC, h)
        assert e.value.status == g.GS_ERR_OOM
    for after in range(4):  # the slab set's per-slab memory, then its contexts' counters
        g.gs_debug_inject_failure(g.GS_INJECT_MALLOC, after)
        with pytest.raises(g.GsError) as e:
            g.gs_slab_create(g.GS_FDTD3D, 16, 16, 16, 2, 1, g.GS_F32, g.GS_BC_PEC, h)
        assert e.value.status == g.GS_ERR_OOM
    for after in range(9):  # the cost model's nine buffers
        g.gs_debug_inject_failure(g.GS_INJECT_MALLOC, after)
        with pytest.raises(g.GsError):
            g.gs_mlp_create(0, h)
    assert _free() == free0
    ctx = g.gs_create(g.GS_FDTD3D, 16, 16, 16, g.GS_F32, g.GS_BC_PEC, h)  # and creation works again
    g.gs_destroy(ctx)


def test_failed_instance_table_allocation_keeps_the_batch_usable():
    import torch

    import paper_2501_09398_gb300 as g

    dims = [(130, 17), (5, 9), (64, 64)]
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=40 + i) for i, (w, h) in enumerate(dims)]
    nx, ny = [d[0] for d in dims], [d[1] for d in dims]
    stream = torch.cuda.Stream()

    def make():
        m = g.gs_multi_create(nx, ny, g.GS_F32, g.GS_BC_CLAMP, stream.cuda_stream)
        bufs = g.MultiFields(m, nx, ny)
        for i, (T, P) in enumerate(fields_np):
            g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
        return m, bufs

    m, bufs = make()
    try:
        g.gs_multi_step(m, 13, 5, g.GS_MULTI_FUSED)
        ref = [g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in enumerate(fields_np)]
    finally:
        g.gs_multi_destroy(m)
        del bufs
    m, bufs = make()
    try:
        g.gs_debug_inject_failure(g.GS_INJECT_MALLOC, 0)
        with pytest.raises(g.GsError) as e:
            g.gs_multi_step(m, 13, 5, g.GS_MULTI_FUSED)
        assert e.value.status == g.GS_ERR_OOM
        assert g.gs_multi_get_parity(m) == 0
        g.gs_multi_step(m, 13, 5, g.GS_MULTI_FUSED)
        got = [g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in enumerate(fields_np)]
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
    finally:
        g.gs_multi_destroy(m)
        del bufs


def test_failed_slab_graph_build_changes_nothing():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(64, 40, 1, seed=22)
    n, S = 23, 5
    base = heat_gpu(T0, P, n, S=0)
    s = g.gs_slab_create(g.GS_HEAT2D, 64, 40, 1, 3, 1, g.GS_F32, g.GS_BC_CLAMP, stream_handle())
    try:
        g.gs_slab_upload(s, g.GS_FIELD_T, T0)
        g.gs_slab_upload(s, g.GS_FIELD_P, P)
        for after in (0, 7, 16):  # nodes of the first and second parity's batch graphs (3 slabs x 5 launches)
            g.gs_debug_inject_failure(g.GS_INJECT_GRAPH_NODE, after)
            with pytest.raises(g.GsError) as e:
                g.gs_slab_step(s, n, S)
            assert e.value.status == g.GS_ERR_CUDA
            got = g.gs_slab_read_field(s, g.GS_FIELD_T, np.empty_like(T0))
            assert np.array_equal(got, T0.astype(np.float32))
            assert g.gs_slab_get_stats(s)["graph_launches"] == 0
        g.gs_slab_step(s, n, S)
        assert np.array_equal(g.gs_slab_read_field(s, g.GS_FIELD_T, np.empty_like(T0)), base)
    finally:
        g.gs_slab_destroy(s)


def test_failed_tuner_snapshot_leaves_the_context_as_it_was():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(96, 64, 1, seed=23)
    base = heat_gpu(T0, P, 20, S=0)
    ctx, fields = heat_setup(96, 64)
    try:
        heat_upload(ctx, T0, P)
        g.gs_debug_inject_failure(g.GS_INJECT_MALLOC, 0)
        with pytest.raises(g.GsError) as e:
            g.gs_autotune(ctx, 10, [({}, 0), ({}, 5)], reps=1)
        assert e.value.status == g.GS_ERR_OOM
        g.gs_step(ctx, 20, 0)
        assert np.array_equal(heat_read(ctx, T0.shape), base)
    finally:
        g.gs_destroy(ctx)
        del fields
