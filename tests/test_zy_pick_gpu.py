"""The pickers on the GPU.

gs_pick: among the workload's candidates that fit its grid, the one whose
mean prediction over the ensemble is smallest.  Checked against the same
candidates scored one model at a time with gs_mlp_predict and reduced on
the host as the library does (the members' float32 predictions summed in
member order, ties to the lowest row).  Untrained models with fitted input
standardisation are enough: the check is of the choice, not of its quality
(the learned picker's regret is checked in test_costmodel_gpu.py).

gs_pick_analytic: the paper's calibrate-fit-minimise on a context, which
must leave the context's fields as they were."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _fitting(g, w):
    out = []
    for plan, S in g.gs_candidates(w):
        try:
            g.gs_plan_check(w, plan)
        except g.GsError:
            continue
        out.append((plan, S))
    return out


@pytest.mark.parametrize("w", [
    dict(kind=1, dtype=0, nx=512, ny=512, nz=8, n_iters=1000),     # 3D thin stack (f32)
    dict(kind=0, dtype=1, nx=4096, ny=4096, nz=1, n_iters=200),    # 2D, bf16
    dict(kind=1, dtype=0, nx=96, ny=80, nz=40, n_iters=300),       # deep stack (no WAVE, no COLUMN_SMEM)
    dict(kind=2, dtype=2, nx=128, ny=128, nz=128, n_iters=5000),   # FDTD, f16
])
def test_pick_is_the_ensembles_argmin(w):
    import torch

    import paper_2501_09398_gb300 as g

    cands = _fitting(g, w)
    assert len(cands) >= 10
    X = g.gs_features(w, cands)
    Xd = torch.from_numpy(X).cuda()
    torch.cuda.synchronize()
    models = [g.gs_mlp_create(seed=s) for s in (3, 4, 5)]
    try:
        preds = []
        for m in models:
            g.gs_mlp_fit_normalization(m, Xd.data_ptr(), X.shape[0])
            out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
            g.gs_mlp_predict(m, Xd.data_ptr(), X.shape[0], out.data_ptr())
            torch.cuda.synchronize()
            preds.append(out.cpu().numpy())
        total = preds[0].copy()
        for p in preds[1:]:
            total = (total + p).astype(np.float32)
        i = int(np.argmin(total))
        plan, S, pred = g.gs_pick(models, w)
        assert (plan, S) == cands[i]
        mean = float(np.float32(total[i]) * np.float32(1.0 / len(models)))
        assert math.isclose(pred, math.exp(mean), rel_tol=1e-5)
        # the single-model ensemble picks that model's own argmin
        plan1, S1, _ = g.gs_pick(models[:1], w)
        assert (plan1, S1) == cands[int(np.argmin(preds[0]))]
    finally:
        for m in models:
            g.gs_mlp_destroy(m)


def test_analytic_pick_on_a_context():
    import torch

    import gs_inputs
    import paper_2501_09398_gb300 as g

    nx, ny, n = 96, 64, 100
    T0, P = gs_inputs.heat_fields(nx, ny, 1, seed=7)
    ctx = g.gs_create(g.GS_HEAT2D, nx, ny, 1, g.GS_F32, g.GS_BC_CLAMP, torch.cuda.Stream().cuda_stream)
    fields = g.HeatFields(ctx, nx, ny, 1)
    try:
        g.gs_upload(ctx, g.GS_FIELD_T, T0)
        g.gs_upload(ctx, g.GS_FIELD_P, P)
        g.gs_step(ctx, 3, 0)  # a state that is not the upload, in buffer T1
        before = g.gs_read_field(ctx, g.GS_FIELD_T, np.empty_like(T0))
        parity = g.gs_get_parity(ctx)
        S, model = g.gs_pick_analytic(ctx, n, reps=1)
        assert S in (1, 10, 50, 100)
        assert all(math.isfinite(model[k]) for k in ("k_c", "b_c", "a", "b"))
        assert g.gs_model_pick(model, [1, 10, 50, 100])[0] == S
        after = g.gs_read_field(ctx, g.GS_FIELD_T, np.empty_like(T0))
        assert np.array_equal(before, after)
        assert g.gs_get_parity(ctx) == parity
        with pytest.raises(g.GsError):
            g.gs_pick_analytic(ctx, 5, reps=1)  # fewer than two batch sizes fit
    finally:
        g.gs_destroy(ctx)
        del fields


@pytest.mark.parametrize("w", [
    dict(kind=1, dtype=0, nx=512, ny=512, nz=8, n_iters=1000),
    dict(kind=0, dtype=0, nx=1024, ny=768, nz=1, n_iters=300),
    dict(kind=2, dtype=1, nx=64, ny=64, nz=64, n_iters=2000),
])
def test_pick_ctx_applies_the_builtin_ensembles_choice(w):
    """gs_pick_ctx with the ensemble compiled into the library equals gs_pick
    with the same members created one by one (gs_mlp_create_builtin), applies
    the chosen plan to the context, and the context then runs it: the result
    of a run with the picked (plan, S) equals a per-step run of the default
    plan bit for bit."""
    import torch

    import gs_inputs
    import paper_2501_09398_gb300 as g

    assert "GB300" in g.gs_mlp_builtin_info()
    models = [g.gs_mlp_create_builtin(k) for k in range(g.GS_MLP_BUILTIN_MEMBERS)]
    try:
        plan_ref, S_ref, pred_ref = g.gs_pick(models, w)
    finally:
        for m in models:
            g.gs_mlp_destroy(m)
    st = torch.cuda.Stream()
    kind, N = w["kind"], w["nx"]
    if kind == g.GS_FDTD3D:
        ctx = g.gs_create(kind, N, N, N, w["dtype"], g.GS_BC_PEC, st.cuda_stream)
        fields = g.FdtdFields(ctx, N, w["dtype"])
        g.gs_set_fdtd_params(ctx, courant=0.5, src_on=1, src=(N // 2,) * 3)
    else:
        ctx = g.gs_create(kind, w["nx"], w["ny"], w["nz"], w["dtype"], g.GS_BC_CLAMP, st.cuda_stream)
        fields = g.HeatFields(ctx, w["nx"], w["ny"], w["nz"], w["dtype"])
    try:
        plan, S, pred = g.gs_pick_ctx(ctx, w["n_iters"])
        assert S == S_ref and math.isclose(pred, pred_ref, rel_tol=1e-6)
        for k in ("block_x", "rows", "temporal_depth", "kernel"):
            assert plan[k] == plan_ref[k], k
        assert g.gs_get_plan(ctx) == plan
        n = 37
        if kind == g.GS_FDTD3D:
            g.gs_step(ctx, n, S)
            got = np.concatenate([g.gs_read_field(ctx, f, np.empty((N + 1,) * 3, np.float32)).ravel()
                                  for f in g.FDTD_FIELDS])
            g.gs_set_plan(ctx)
            z = np.zeros((N + 1,) * 3, dtype=np.float32)
            for f in g.FDTD_FIELDS:
                g.gs_upload(ctx, f, z)
            g.gs_set_time(ctx, 0)
            g.gs_step(ctx, n, 0)
            ref = np.concatenate([g.gs_read_field(ctx, f, np.empty((N + 1,) * 3, np.float32)).ravel()
                                  for f in g.FDTD_FIELDS])
        else:
            T0, P = gs_inputs.heat_fields(w["nx"], w["ny"], w["nz"], seed=5)
            g.gs_upload(ctx, g.GS_FIELD_T, T0)
            g.gs_upload(ctx, g.GS_FIELD_P, P)
            g.gs_step(ctx, n, S)
            got = g.gs_read_field(ctx, g.GS_FIELD_T, np.empty_like(T0))
            g.gs_set_plan(ctx)
            g.gs_set_parity(ctx, 0)
            g.gs_upload(ctx, g.GS_FIELD_T, T0)
            g.gs_step(ctx, n, 0)
            ref = g.gs_read_field(ctx, g.GS_FIELD_T, np.empty_like(T0))
        assert np.array_equal(got, ref)
    finally:
        g.gs_destroy(ctx)
        del fields


@pytest.mark.parametrize("N", [40, 128, 256])
def test_pick_ctx_in_media_takes_a_plan_media_run_on(N):
    # an FDTD context with a media table: the pick is among the plans media
    # run on (COLUMN, the fused march), never the k-march kernels, and the
    # context steps with it, bit for bit as the per-step COLUMN launches
    import gs_inputs
    import paper_2501_09398_gb300 as g
    from gsutil import FDTD_NAMES, fdtd_read, fdtd_setup, fdtd_upload

    media = gs_inputs.fdtd_media(N, n_mat=4, n_boxes=6, seed=N)
    init = gs_inputs.fdtd_random_all(N, seed=N + 1)
    src, n = (N // 2, N // 3, N // 2), 9
    outs = []
    for pick in (True, False):
        ctx, fields = fdtd_setup(N, "f32", None, src, media=media)
        try:
            fdtd_upload(ctx, N, init)
            if pick:
                plan, S, pred = g.gs_pick_ctx(ctx, 1000)
                assert plan["kernel"] == g.GS_KERNEL_COLUMN or \
                    (plan["kernel"] == g.GS_KERNEL_FUSED and plan["tile_y"] >= 1), plan
                assert math.isfinite(pred) and pred > 0
            else:
                S = 0
            g.gs_step(ctx, n, S)
            outs.append(fdtd_read(ctx, N))
        finally:
            g.gs_destroy(ctx)
            del fields
    assert all(np.array_equal(outs[0][k], outs[1][k]) for k in FDTD_NAMES)


def test_pick_ctx_refuses_a_skeleton_context():
    import paper_2501_09398_gb300 as g

    ctx = g.gs_create(g.GS_SKELETON, 1000, 1, 1)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_pick_ctx(ctx, 100)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
    finally:
        g.gs_destroy(ctx)


def test_measured_regret_of_the_builtin_ensemble():
    """The learned pick checked by running it: whole runs (graph creation
    included, median of five) of 15 held-out workloads of the packaged sweep,
    five of each kind, with the compiled-in ensemble's pick, the sweep's best
    candidate and the analytic pick; the learned pick's measured mean regret
    against the fastest of the three stays within 5 %.  The contexts run on
    one explicit stream, the one the timing events are recorded on."""
    from paper_2501_09398_gb300 import costmodel as cm
    from paper_2501_09398_gb300 import gs_mlp_destroy

    _, held = cm.load_tables()
    models = cm.builtin_models()
    try:
        recs = cm.measured_regret(models, held, n=15, seed=11, reps=5, max_run_ms=150.0)
    finally:
        for m in models:
            gs_mlp_destroy(m)
    s = cm.summarize_measured(recs)
    print({k: v for k, v in s.items()})
    assert s["workloads"] == 15
    assert s["learned"]["mean"] <= 0.05
