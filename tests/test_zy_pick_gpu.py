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
