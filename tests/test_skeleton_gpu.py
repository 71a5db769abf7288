"""The paper's skeleton application (in-place vector scale, Sec. III-C) on
the GPU: closed forms, FP64 oracle parity, graph vs per-step bit-identity,
and calibration of the paper's model (Eqs. 2 and 6) on it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _run(x0, c, n, S, dtype=0, plan=None):
    import torch

    import paper_2501_09398_gb300 as g

    ctx = g.gs_create(g.GS_SKELETON, x0.size, 1, 1, dtype, g.GS_BC_CLAMP, None)
    pitch = g.gs_required_pitch(dtype, x0.size)
    buf = torch.zeros(pitch, dtype={0: torch.float32, 1: torch.bfloat16, 2: torch.float16}[dtype], device="cuda")
    torch.cuda.synchronize()
    try:
        g.gs_bind_field(ctx, g.GS_FIELD_X, buf.data_ptr(), pitch)
        g.gs_set_scale(ctx, c)
        if plan:
            g.gs_set_plan(ctx, **plan)
        g.gs_upload(ctx, g.GS_FIELD_X, np.ascontiguousarray(x0, dtype=np.float32))
        g.gs_step(ctx, n, S)
        return g.gs_read_field(ctx, g.GS_FIELD_X, np.empty(x0.size, dtype=np.float32))
    finally:
        g.gs_destroy(ctx)


@pytest.mark.parametrize("size", [1, 7, 1000, 4099, 1_000_000])
def test_skeleton_parity(oracle, size):
    rng = np.random.default_rng(size)
    x0 = rng.uniform(-2, 2, size).astype(np.float32)
    assert np.array_equal(_run(x0, -1.0, 9, 4), -x0)  # exact: (-1)^9
    c, n = 1.0 + 2.0 ** -8, 300
    got = _run(x0, c, n, 100)
    ref = oracle.skeleton_run(x0, c, n)
    # one FP32 rounding per iteration: relative error <= n * 2^-24
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= n * 2.0 ** -24
    for S, plan in ((0, None), (7, None), (300, dict(use_pdl=1)), (64, dict(device_launch=1)), (5, dict(block_x=64))):
        assert np.array_equal(_run(x0, c, n, S, plan=plan), got), (S, plan)


def test_skeleton_model_calibration():
    import torch

    import paper_2501_09398_gb300 as g

    n = 1000
    ctx = g.gs_create(g.GS_SKELETON, n, 1, 1, g.GS_F32, g.GS_BC_CLAMP, None)
    buf = torch.ones(n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    try:
        g.gs_bind_field(ctx, g.GS_FIELD_X, buf.data_ptr(), n)
        m = g.gs_model_calibrate(ctx, 1000, [1, 10, 50, 100, 500, 1000], reps=2)
        assert m["k_c"] > 0 and m["a"] > 0, m  # creation grows with S; Obs. I: T_i < T_a
    finally:
        g.gs_destroy(ctx)
