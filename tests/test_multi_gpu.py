"""Uneven instance batches: the fused persistent kernel (per-step and in
stream-captured graphs) against per-instance launches and the FP64 oracle."""
import numpy as np
import pytest

import gs_inputs
from gsutil import HEAT_RTOL, max_rel, stream_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _run(sides, fields_np, n, S, mode, plan=None, stream=None, dims=None):
    import torch

    import paper_2501_09398_gb300 as g

    nx = [d[0] for d in dims] if dims else sides
    ny = [d[1] for d in dims] if dims else sides
    if stream is None:
        stream = torch.cuda.Stream()
    m = g.gs_multi_create(nx, ny, g.GS_F32, g.GS_BC_CLAMP, stream.cuda_stream)
    bufs = g.MultiFields(m, nx, ny)
    try:
        if plan:
            g.gs_multi_set_plan(m, **plan)
        for i, (T, P) in enumerate(fields_np):
            g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
        g.gs_multi_step(m, n, S, mode)
        out = [g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in enumerate(fields_np)]
        return out, g.gs_multi_get_stats(m)
    finally:
        g.gs_multi_destroy(m)
        del bufs


def test_small_batch_all_modes_bit_identical(oracle):
    import paper_2501_09398_gb300 as g

    dims = [(130, 17), (5, 9), (64, 64), (200, 3), (1, 1), (77, 120)]
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=300 + i) for i, (w, h) in enumerate(dims)]
    n = 23
    base, _ = _run(None, fields_np, n, 0, g.GS_MULTI_SEPARATE, dims=dims)
    for i, (T, P) in enumerate(fields_np):
        assert max_rel(base[i], oracle.heat_run(T, P, n, oracle.HEAT_COEFFS_2D)) <= HEAT_RTOL
    for S, mode, plan in ((0, g.GS_MULTI_FUSED, None), (7, g.GS_MULTI_FUSED, None), (23, g.GS_MULTI_FUSED, None),
                          (5, g.GS_MULTI_FUSED, dict(block_x=32, rows=3, blocks=7, kernel=g.GS_KERNEL_MARCH)),
                          (5, g.GS_MULTI_FUSED, dict(rows=8, blocks=5, kernel=g.GS_KERNEL_COLUMN)),
                          (0, g.GS_MULTI_FUSED, dict(rows=1, kernel=g.GS_KERNEL_COLUMN)),
                          (4, g.GS_MULTI_FUSED, dict(use_pdl=1)), (6, g.GS_MULTI_SEPARATE, None)):
        got, st = _run(None, fields_np, n, S, mode, plan=plan, dims=dims)
        assert all(np.array_equal(a, b) for a, b in zip(got, base)), (S, mode, plan)
        if mode == g.GS_MULTI_FUSED and S > 0:
            assert st["graph_launches"] == n // S + (1 if n % S else 0)


@pytest.mark.parametrize("depth", [2, 4])
def test_temporal_depth_bit_identical(depth):
    # each fused launch advances every instance `depth` steps with the
    # temporally blocked COLUMN tile; n mod depth steps run at depth 1
    import paper_2501_09398_gb300 as g

    dims = [(130, 17), (5, 9), (64, 64), (200, 3), (1, 1), (77, 120), (300, 41)]
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=350 + i) for i, (w, h) in enumerate(dims)]
    n = 23
    base, _ = _run(None, fields_np, n, 0, g.GS_MULTI_SEPARATE, dims=dims)
    for S, plan in ((0, dict(rows=4)), (7, dict(rows=2)), (8, dict(rows=8, blocks=5)), (23, dict(rows=1)),
                    (5, dict(rows=4, traverse=g.GS_TRAVERSE_ALTERNATE))):
        plan = dict(plan, kernel=g.GS_KERNEL_COLUMN, temporal_depth=depth)
        got, st = _run(None, fields_np, n, S, g.GS_MULTI_FUSED, plan=plan, dims=dims)
        assert all(np.array_equal(a, b) for a, b in zip(got, base)), (S, plan)
        if S == 0:
            assert st["kernel_launches"] == n // depth + n % depth


def test_temporal_depth_plan_errors():
    import torch

    import paper_2501_09398_gb300 as g

    m = g.gs_multi_create([16, 8], [16, 8], g.GS_F32, g.GS_BC_CLAMP, torch.cuda.Stream().cuda_stream)
    try:
        with pytest.raises(g.GsError):
            g.gs_multi_set_plan(m, kernel=g.GS_KERNEL_MARCH, temporal_depth=2)
        with pytest.raises(g.GsError):
            g.gs_multi_set_plan(m, kernel=g.GS_KERNEL_COLUMN, temporal_depth=3)
        g.gs_multi_set_plan(m, kernel=g.GS_KERNEL_COLUMN, temporal_depth=4)
    finally:
        g.gs_multi_destroy(m)


def test_unbound_instance_is_a_state_error():
    import torch

    import paper_2501_09398_gb300 as g

    m = g.gs_multi_create([16, 8], [16, 8], g.GS_F32, g.GS_BC_CLAMP, torch.cuda.Stream().cuda_stream)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_multi_step(m, 3, 0, g.GS_MULTI_FUSED)
        assert e.value.status == g.GS_ERR_STATE
        with pytest.raises(g.GsError) as e:
            g.gs_multi_bind_field(m, 5, g.GS_FIELD_T0, 0, 16)
        assert e.value.status == g.GS_ERR_INVALID_ARG
    finally:
        g.gs_multi_destroy(m)


def test_config3_batch(oracle):
    # 64 square grids, sides log-uniform in [64, 1024], seeds 1000+k, 2000 iterations
    import paper_2501_09398_gb300 as g

    sides = gs_inputs.instance_sides(64, 64, 1024, seed=0)
    fields_np = gs_inputs.instance_fields(sides)
    n = 2000
    fused, _ = _run(sides, fields_np, n, 100, g.GS_MULTI_FUSED)
    sep, _ = _run(sides, fields_np, n, 0, g.GS_MULTI_SEPARATE)
    assert all(np.array_equal(a, b) for a, b in zip(fused, sep))
    # the bench's plan: fused launches of temporal depth 2, COLUMN tiles of 2 rows
    fused2, _ = _run(sides, fields_np, n, 100, g.GS_MULTI_FUSED,
                     plan=dict(kernel=g.GS_KERNEL_COLUMN, rows=2, temporal_depth=2))
    assert all(np.array_equal(a, b) for a, b in zip(fused2, sep))
    order = np.argsort(sides)
    for i in list(order[:6]) + [order[-1]]:
        T, P = fields_np[i]
        err = max_rel(fused[i], oracle.heat_run(T, P, n, oracle.HEAT_COEFFS_2D))
        assert err <= HEAT_RTOL, (i, sides[i], err)


def test_multi_autotune_restores_state_and_returns_its_argmin():
    """gs_multi_autotune over the library's candidate list: every candidate
    runs (or is skipped with its status), the best index is the argmin of
    the returned totals, and the batch's fields, parity and plan are as they
    were (a step after tuning equals a step of an untuned batch)."""
    import torch

    import paper_2501_09398_gb300 as g

    dims = [(130, 17), (5, 9), (64, 64), (200, 3), (77, 120), (300, 40)]
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=700 + i) for i, (w, h) in enumerate(dims)]
    nx, ny = [d[0] for d in dims], [d[1] for d in dims]
    stream = torch.cuda.Stream()
    ref, _ = _run(None, fields_np, 7 + 30, 0, g.GS_MULTI_FUSED, stream=stream, dims=dims)

    m = g.gs_multi_create(nx, ny, g.GS_F32, g.GS_BC_CLAMP, stream.cuda_stream)
    bufs = g.MultiFields(m, nx, ny)
    try:
        for i, (T, P) in enumerate(fields_np):
            g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
        g.gs_multi_step(m, 7, 0, g.GS_MULTI_FUSED)  # odd: the state sits in T1
        plan0 = g.gs_multi_get_plan(m)
        cands = g.gs_multi_candidates(m)
        assert len(cands) == 56 and all(S in (0, 10, 100, 1000) for _, S in cands)
        res, best = g.gs_multi_autotune(m, 30, cands, reps=2)
        ok = [i for i, r in enumerate(res) if r["status"] == g.GS_OK]
        assert len(ok) == len(cands)  # every candidate of the list runs on these grids
        assert best == min(ok, key=lambda i: res[i]["total_ms"])
        for r, (plan, S) in zip(res, cands):
            assert r["batch_size"] == S and r["exec_ms_per_iter"] > 0
            assert (r["build_seconds"] > 0) == (S > 0)
            for k in ("kernel", "rows", "temporal_depth"):
                assert r["plan"][k] == plan[k]
        assert g.gs_multi_get_plan(m) == plan0 and g.gs_multi_get_parity(m) == 1
        g.gs_multi_step(m, 30, 0, g.GS_MULTI_FUSED)
        got = [g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in enumerate(fields_np)]
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        # the tuned plan runs bit-identically too
        g.gs_multi_set_plan(m, **res[best]["plan"])
    finally:
        g.gs_multi_destroy(m)
        del bufs
