"""The fused FDTD step (GS_KERNEL_FUSED: H and E of a Yee step in one
launch, out of place into a second, library-owned set of the six
components, steps in pairs so the state ends in the bound fields, an odd
last step as the in-place H and E launches), in its column form and
marching planes in k (plan.tile_y >= 1): bit-identical to the
two-launch step from random values in every entry (walls included), with
sources on the walls and the aligned layout's i = N column, per-step and in
graph batches with peeled remainders, in every storage type; and against
the FP64 oracle on the 128^3 driven cavity after 5000 steps."""
import numpy as np
import pytest

import gs_inputs
from gsutil import FDTD_NAMES, FDTD_RL2, fdtd_concat, fdtd_read, fdtd_setup, fdtd_upload, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _run(N, n, S, src, init, plan=None, dtype="f32", steps=None):
    import paper_2501_09398_gb300 as g

    ctx, fields = fdtd_setup(N, dtype, plan, src)
    try:
        fdtd_upload(ctx, N, init)
        for part in (steps or [n]):
            g.gs_step(ctx, part, S)
        out = fdtd_read(ctx, N)
        return out, g.gs_get_time(ctx), g.gs_get_stats(ctx)
    finally:
        g.gs_destroy(ctx)
        del fields


@pytest.mark.parametrize("N,src", [(9, (4, 4, 4)), (16, (16, 8, 3)), (33, (0, 16, 16)), (37, (37, 20, 20)),
                                   (128, (128, 64, 64)), (128, (64, 0, 127))])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_fused_bit_identical_to_two_launches(N, src, dtype):
    import paper_2501_09398_gb300 as g

    init = gs_inputs.fdtd_random_all(N, seed=N + 1)
    n = 13 if N < 100 else 5
    base, t0, _ = _run(N, n, 0, src, init, dtype=dtype)
    # tile_y 0: the column form; tile_y >= 1: blocks march tile_y planes in k
    for S, rows, tile_y in ((0, 2, 0), (4, 1, 0), (6, 8, 0), (13, 4, 0),
                            (0, 2, 1), (4, 1, 3), (6, 8, 7), (13, 4, 1000)):
        plan = dict(kernel=g.GS_KERNEL_FUSED, rows=rows, tile_y=tile_y)
        got, t, st = _run(N, n, S, src, init, plan=plan, dtype=dtype)
        assert t == t0 == n
        for k in FDTD_NAMES:
            assert np.array_equal(got[k], base[k]), (S, rows, tile_y, k)
    # resume across calls of odd length (each call ends in the bound fields)
    got, t, _ = _run(N, n, 3, src, init, plan=dict(kernel=g.GS_KERNEL_FUSED), dtype=dtype, steps=[5, n - 5])
    assert t == n and all(np.array_equal(got[k], base[k]) for k in FDTD_NAMES)


def test_fused_launch_counts():
    import paper_2501_09398_gb300 as g

    N = 16
    init = gs_inputs.fdtd_random_all(N, seed=3)
    _, _, st = _run(N, 9, 0, (8, 8, 8), init, plan=dict(kernel=g.GS_KERNEL_FUSED))
    assert st["kernel_launches"] == 8 + 2  # four fused pairs, then the odd step's H and E


def test_fused_config2_full_size(fdtd_config2_ref):
    import paper_2501_09398_gb300 as g

    got, _, _ = _run(128, 5000, 100, (64, 64, 64), {}, plan=dict(kernel=g.GS_KERNEL_FUSED))
    err = rel_l2(fdtd_concat(got), fdtd_concat(fdtd_config2_ref))
    print(f"config2 fused f32 rel L2 {err:.3e}")
    assert err <= FDTD_RL2


def test_fused_march_config2_full_size(fdtd_config2_ref):
    import paper_2501_09398_gb300 as g

    got, _, _ = _run(128, 5000, 100, (64, 64, 64), {}, plan=dict(kernel=g.GS_KERNEL_FUSED, rows=8, tile_y=16))
    err = rel_l2(fdtd_concat(got), fdtd_concat(fdtd_config2_ref))
    print(f"config2 fused march f32 rel L2 {err:.3e}")
    assert err <= FDTD_RL2


def test_fused_refusals():
    import paper_2501_09398_gb300 as g

    h = None
    ctx = g.gs_create(g.GS_HEAT2D, 32, 32, 1)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_set_plan(ctx, kernel=g.GS_KERNEL_FUSED)
        assert e.value.status == g.GS_ERR_INVALID_ARG
    finally:
        g.gs_destroy(ctx)
    ctx = g.gs_create(g.GS_FDTD3D, 16, 16, 16, g.GS_F32, g.GS_BC_PEC)
    try:
        for ty in (-1, (1 << 20) + 1):
            with pytest.raises(g.GsError) as e:
                g.gs_set_plan(ctx, kernel=g.GS_KERNEL_FUSED, tile_y=ty)
            assert e.value.status == g.GS_ERR_INVALID_ARG
    finally:
        g.gs_destroy(ctx)
    # media run on the two-launch column kernels
    N = 16
    mat, table = gs_inputs.fdtd_media(N, n_mat=3, n_boxes=4, seed=1)
    ctx, fields = fdtd_setup(N, "f32", dict(kernel=g.GS_KERNEL_FUSED), (8, 8, 8), media=(mat, table))
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_step(ctx, 2, 0)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
    finally:
        g.gs_destroy(ctx)
        del fields
    s = g.gs_slab_create(g.GS_FDTD3D, 16, 16, 16, 2, 1, g.GS_F32, g.GS_BC_PEC, h)
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_slab_set_plan(s, kernel=g.GS_KERNEL_FUSED)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
    finally:
        g.gs_slab_destroy(s)
