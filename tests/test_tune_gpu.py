"""Autotuner: every runnable candidate is timed, unrunnable ones are skipped
with their status, the argmin of T_C + T_E is returned, and the context's
fields, parity and plan are left as they were."""
import numpy as np
import pytest

import gs_inputs
from gsutil import heat_read, heat_setup, heat_upload, fdtd_read, fdtd_setup, fdtd_upload, FDTD_NAMES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def test_autotune_thermal_restores_state():
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(200, 120, 1, seed=31)
    ctx, fields = heat_setup(200, 120)
    try:
        heat_upload(ctx, T0, P)
        g.gs_step(ctx, 3, 0)  # parity 1, some state
        before = heat_read(ctx, T0.shape)
        plan_before = g.gs_get_plan(ctx)
        cands = [(dict(), 0), (dict(), 10), (dict(block_x=64, rows=4), 25), (dict(temporal_depth=3), 10),
                 (dict(temporal_depth=4, kernel=g.GS_KERNEL_WAVE, rows=8, block_x=64), 20),
                 (dict(temporal_depth=2, kernel=g.GS_KERNEL_TILE, tile_x=32, tile_y=16), 50)]
        res, best = g.gs_autotune(ctx, 50, cands, reps=2)
        assert [r["status"] for r in res] == [0, 0, 0, g.GS_ERR_INVALID_ARG, 0, 0]
        ok = [i for i, r in enumerate(res) if r["status"] == 0]
        assert best in ok
        assert res[best]["total_ms"] == min(res[i]["total_ms"] for i in ok)
        assert res[0]["build_seconds"] == 0 and all(res[i]["build_seconds"] > 0 for i in (1, 2, 4, 5))
        assert all(res[i]["exec_ms_per_iter"] > 0 for i in ok)
        assert g.gs_get_parity(ctx) == 1
        assert g.gs_get_plan(ctx) == plan_before
        assert np.array_equal(heat_read(ctx, T0.shape), before)
        # stepping continues exactly as if the tuner had not run
        g.gs_step(ctx, 4, 2)
        ref_ctx, ref_fields = heat_setup(200, 120)
        heat_upload(ref_ctx, T0, P)
        g.gs_step(ref_ctx, 7, 0)
        assert np.array_equal(heat_read(ctx, T0.shape), heat_read(ref_ctx, T0.shape))
        g.gs_destroy(ref_ctx)
    finally:
        g.gs_destroy(ctx)
        del fields


def test_autotune_fdtd_restores_time():
    import paper_2501_09398_gb300 as g

    N = 16
    ctx, fields = fdtd_setup(N, src=(8, 8, 8))
    try:
        fdtd_upload(ctx, N, {})
        g.gs_step(ctx, 30, 0)
        before = fdtd_read(ctx, N)
        res, best = g.gs_autotune(ctx, 40, [(dict(), 0), (dict(rows=4), 8), (dict(block_x=64, rows=32), 40)], reps=1)
        assert best in (0, 1, 2) and all(r["status"] == 0 for r in res)
        assert g.gs_get_time(ctx) == 30
        after = fdtd_read(ctx, N)
        assert all(np.array_equal(before[k], after[k]) for k in FDTD_NAMES)
    finally:
        g.gs_destroy(ctx)
        del fields


def test_autotune_needs_bound_fields():
    import paper_2501_09398_gb300 as g

    ctx = g.gs_create(g.GS_HEAT2D, 32, 32, 1, g.GS_F32, g.GS_BC_CLAMP, None)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_autotune(ctx, 10, [(dict(), 0)])
        assert e.value.status == g.GS_ERR_STATE
    finally:
        g.gs_destroy(ctx)


def test_model_calibrate_on_gpu():
    # Fit Eqs. 2 and 6 on a small 2D grid.  Graph creation grows with the
    # node count (k_c > 0), and on GB300 the time between nodes inside a
    # graph is shorter than between graph launches (Obs. I: a > 0).
    import paper_2501_09398_gb300 as g

    T0, P = gs_inputs.heat_fields(256, 256, 1, seed=33)
    ctx, fields = heat_setup(256, 256)
    try:
        heat_upload(ctx, T0, P)
        before = heat_read(ctx, T0.shape)
        m = g.gs_model_calibrate(ctx, 1000, [1, 10, 50, 100, 500, 1000], reps=2)
        assert all(np.isfinite(v) for v in m.values())
        assert m["k_c"] > 0 and m["a"] > 0, m
        best, total = g.gs_model_pick(m, [1, 10, 50, 100, 500, 1000])
        assert best in (10, 50, 100, 500, 1000)
        assert np.array_equal(heat_read(ctx, T0.shape), before)
    finally:
        g.gs_destroy(ctx)
        del fields
