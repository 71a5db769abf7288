"""GPU parity of the Yee FDTD kernels against the FP64 oracle, through the C
ABI: the source-driven cavity (relative L2 over all six components
concatenated <= 1e-4), energy invariance and cavity-mode dispersion of the
FP32 kernels, bit-identity of per-step vs graph-batched runs, and the device
step counter that feeds the source."""
import math

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


def _gpu_run(N, n, S, src=None, init=None, plan=None, dtype="f32"):
    import paper_2501_09398_gb300 as g

    ctx, fields = fdtd_setup(N, dtype, plan, src)
    try:
        fdtd_upload(ctx, N, init or {})
        g.gs_step(ctx, n, S)
        return fdtd_read(ctx, N)
    finally:
        g.gs_destroy(ctx)
        del fields


def _oracle_run(oracle, N, n, src=None, init=None):
    f = oracle.fdtd_zero_fields(N)
    for k, v in (init or {}).items():
        f[k][...] = np.asarray(v, dtype=np.float64)
    return oracle.fdtd_run(f, N, n, courant=0.5, src=src)


@pytest.mark.parametrize("N", [9, 16, 33])
def test_driven_cavity_parity_small(oracle, N):
    c = N // 2
    n = 150
    ref = _oracle_run(oracle, N, n, src=(c, c, c))
    got = _gpu_run(N, n, 0, src=(c, c, c))
    err = rel_l2(fdtd_concat(got), fdtd_concat(ref))
    assert err <= FDTD_RL2, err
    # Per component, measured against the whole field's norm: the source
    # leaves a large static E, and H (orders of magnitude smaller) is a
    # difference of nearly equal E values, so its own relative error
    # reflects FP32 cancellation (plain FP32 arithmetic shows the same).
    total = np.linalg.norm(fdtd_concat(ref))
    for name in FDTD_NAMES:
        assert np.linalg.norm(got[name].astype(np.float64) - ref[name]) <= FDTD_RL2 * total, name


def test_graph_bit_identical_and_plans():
    N = 20
    src = (7, 11, 5)
    base = _gpu_run(N, 45, 0, src=src)
    for S in (1, 4, 7, 45, 60):
        got = _gpu_run(N, 45, S, src=src)
        assert all(np.array_equal(got[k], base[k]) for k in FDTD_NAMES), f"S={S}"
    import paper_2501_09398_gb300 as g

    for plan in (dict(use_pdl=1), dict(rows=1), dict(rows=3), dict(rows=8), dict(device_launch=1),
                 dict(kernel=g.GS_KERNEL_MARCH, block_x=32, rows=3),
                 dict(kernel=g.GS_KERNEL_MARCH, block_x=128, rows=40)):
        got = _gpu_run(N, 45, 9, src=src, plan=plan)
        assert all(np.array_equal(got[k], base[k]) for k in FDTD_NAMES), str(plan)


def test_random_field_parity_and_energy(oracle):
    # source-free PEC cavity from a random interior E field
    N = 24
    e0 = gs_inputs.fdtd_random_e(N, seed=4)
    ref = _oracle_run(oracle, N, 300, init=e0)
    got = _gpu_run(N, 300, 25, init=e0)
    assert rel_l2(fdtd_concat(got), fdtd_concat(ref)) <= FDTD_RL2


def test_energy_invariant_on_gpu():
    # W^m = |E^m|^2 + H^{m-1/2}.H^{m+1/2} is exactly invariant for the
    # scheme; FP32 rounding lets it drift by ~1e-6 over a few thousand steps.
    import paper_2501_09398_gb300 as g

    N = 24
    e0 = gs_inputs.fdtd_random_e(N, seed=5)
    ctx, fields = fdtd_setup(N)
    try:
        fdtd_upload(ctx, N, e0)  # H^{-1/2} = 0
        W = []
        for m in (0, 499, 1999):
            g.gs_step(ctx, m - g.gs_get_time(ctx), 100)
            cur = fdtd_read(ctx, N)  # E^m, H^{m-1/2}
            g.gs_step(ctx, 1, 0)
            nxt = fdtd_read(ctx, N)  # H^{m+1/2}
            e2 = sum(float(np.sum(cur[k].astype(np.float64) ** 2)) for k in ("Ex", "Ey", "Ez"))
            hh = sum(float(np.sum(cur[k].astype(np.float64) * nxt[k].astype(np.float64))) for k in ("Hx", "Hy", "Hz"))
            W.append(e2 + hh)
        assert max(abs(w - W[0]) for w in W) <= 1e-5 * W[0], W
    finally:
        g.gs_destroy(ctx)
        del fields


def test_cavity_mode_dispersion_on_gpu():
    import paper_2501_09398_gb300 as g

    N, s = 32, 0.5
    idx = np.arange(N + 1)
    mode = np.zeros((N + 1,) * 3)
    mode[:N, :, :] = np.outer(np.sin(math.pi * idx / N), np.sin(math.pi * idx / N))[None]
    ctx, fields = fdtd_setup(N)
    try:
        fdtd_upload(ctx, N, {"Ez": mode.astype(np.float32)})
        a = []
        for _ in range(30):
            f = fdtd_read(ctx, N)
            a.append(float(np.sum(f["Ez"].astype(np.float64) * mode)))
            g.gs_step(ctx, 1, 0)
        cos_pred = 1.0 - 2.0 * s * s * 2.0 * math.sin(math.pi / (2 * N)) ** 2
        amp = max(abs(v) for v in a)
        est = [(a[n + 1] + a[n - 1]) / (2 * a[n]) for n in range(1, len(a) - 1) if abs(a[n]) > 0.3 * amp]
        assert est and max(abs(e - cos_pred) for e in est) <= 2e-6
    finally:
        g.gs_destroy(ctx)
        del fields


def test_step_counter_and_resume():
    import paper_2501_09398_gb300 as g

    N, src = 12, (6, 6, 6)
    full = _gpu_run(N, 80, 10, src=src)
    ctx, fields = fdtd_setup(N, src=src)
    try:
        fdtd_upload(ctx, N, {})
        g.gs_step(ctx, 33, 10)
        mid = fdtd_read(ctx, N)
        assert g.gs_get_time(ctx) == 33
        g.gs_destroy(ctx)
        ctx = None
        ctx2, fields2 = fdtd_setup(N, src=src)
        fdtd_upload(ctx2, N, mid)
        g.gs_set_time(ctx2, 33)  # the source resumes at n = 33
        g.gs_step(ctx2, 47, 10)
        got = fdtd_read(ctx2, N)
        assert all(np.array_equal(got[k], full[k]) for k in FDTD_NAMES)
        g.gs_destroy(ctx2)
        del fields2
    finally:
        if ctx is not None:
            g.gs_destroy(ctx)
        del fields


def test_config2_full_size(fdtd_config2_ref):
    # 128^3 cells, courant 0.5, PEC, soft Ez source at the centre, 5000 steps
    N, n = 128, 5000
    src = (64, 64, 64)
    ref = fdtd_config2_ref
    got = _gpu_run(N, n, 100, src=src)
    err = rel_l2(fdtd_concat(got), fdtd_concat(ref))
    print(f"config2 f32 rel L2 {err:.3e}")
    assert err <= FDTD_RL2


@pytest.mark.parametrize("N,src", [(128, (128, 64, 64)), (128, (64, 0, 64)), (37, (37, 20, 20))])
def test_wall_column_and_wall_source(oracle, N, src):
    # N = 128: the warps tile i in [0, N) exactly and lane 31 updates the
    # i = N column (Hx) as an extra cell; from random values in every entry
    # (walls included) Hx there changes every step.  A source on the i = N
    # wall or on the j = 0 wall exercises the extra-cell and boundary-row
    # source paths and the step counter.  N = 37 is the ragged layout.
    n = 12
    init = gs_inputs.fdtd_random_all(N, seed=N)
    ref = _oracle_run(oracle, N, n, src=src, init=init)
    got = _gpu_run(N, n, 5, src=src, init=init)
    assert rel_l2(fdtd_concat(got), fdtd_concat(ref)) <= FDTD_RL2
    wall = got["Hx"][:, :, N].astype(np.float64)
    ref_wall = ref["Hx"][:, :, N]
    assert np.linalg.norm(wall - ref_wall) <= FDTD_RL2 * np.linalg.norm(ref_wall)
    assert np.linalg.norm(ref_wall - init["Hx"][:, :, N]) > 0.1 * np.linalg.norm(ref_wall)
    si, sj, sk = src
    assert abs(float(got["Ez"][sk, sj, si]) - ref["Ez"][sk, sj, si]) <= 1e-5 * (1.0 + abs(ref["Ez"][sk, sj, si]))
    per_step = _gpu_run(N, n, 0, src=src, init=init)
    assert all(np.array_equal(got[k], per_step[k]) for k in FDTD_NAMES)


@pytest.mark.parametrize("src", [(128, 128, 128), (256, 100, 100), (127, 40, 200)])
def test_two_blocks_along_i_aligned(oracle, src):
    # N = 256: the aligned layout with two blocks along i.  Only the last
    # block's lane 31 owns the extra i = N cell; the lanes 31 of the first
    # block end where the second block's lane 0 begins (i = 128), which must
    # be updated, and fed by the source, exactly once.  From random values
    # in every entry, against the oracle, with the step counter; the fused
    # step (column form and k march) bit-identical to the two launches.
    import paper_2501_09398_gb300 as g

    N, n = 256, 6
    init = gs_inputs.fdtd_random_all(N, seed=11)
    ref = _oracle_run(oracle, N, n, src=src, init=init)
    ctx, fields = fdtd_setup(N, "f32", dict(kernel=g.GS_KERNEL_COLUMN, rows=2), src)
    try:
        fdtd_upload(ctx, N, init)
        g.gs_step(ctx, n, 4)
        got = fdtd_read(ctx, N)
        assert g.gs_get_time(ctx) == n
    finally:
        g.gs_destroy(ctx)
        del fields
    assert rel_l2(fdtd_concat(got), fdtd_concat(ref)) <= FDTD_RL2
    for name in FDTD_NAMES:  # the block seam i = 128 and the i = N column, element by element
        for i in (127, 128, N):
            d = np.abs(got[name][:, :, i].astype(np.float64) - ref[name][:, :, i])
            assert np.all(d <= 1e-5 * (1.0 + np.abs(ref[name][:, :, i]))), (name, i)
    for plan in (dict(kernel=g.GS_KERNEL_FUSED, rows=8), dict(kernel=g.GS_KERNEL_FUSED, rows=8, tile_y=32)):
        fused = _gpu_run(N, n, 4, src=src, init=init, plan=plan)
        assert all(np.array_equal(fused[k], got[k]) for k in FDTD_NAMES), plan


def test_driven_energy_budget_on_gpu():
    # the soft source's exact discrete energy budget on the GPU's own FP32
    # fields, one step at a time: W^{n+1} - W^n = g(n) (Ez^{n+1} + Ez^n)[src]
    import paper_2501_09398_gb300 as g

    N, amp, delay, width = 24, 0.8, 20.0, 8.0
    si, sj, sk = src = (12, 11, 13)
    ctx, fields = fdtd_setup(N)
    E, H = ("Ex", "Ey", "Ez"), ("Hx", "Hy", "Hz")
    try:
        g.gs_set_fdtd_params(ctx, courant=0.5, src_on=1, src=src, amp=amp, delay=delay, width=width)
        fdtd_upload(ctx, N, {})
        g.gs_set_time(ctx, 0)
        hist = [fdtd_read(ctx, N)]
        for _ in range(46):
            g.gs_step(ctx, 1, 0)
            hist.append(fdtd_read(ctx, N))
    finally:
        g.gs_destroy(ctx)
        del fields
    h = [{c: np.zeros_like(hist[0][c], dtype=np.float64) for c in H}] + [
        {c: f[c].astype(np.float64) for c in H} for f in hist[1:]]  # h[n] = H^{n-1/2}
    e = [{c: f[c].astype(np.float64) for c in E} for f in hist]
    W = [sum(float(np.sum(e[n][c] ** 2)) for c in E) + sum(float(np.sum(h[n][c] * h[n + 1][c])) for c in H)
         for n in range(45)]
    scale = max(abs(w) for w in W)
    assert scale > 1.0
    for n in range(44):
        gn = amp * math.exp(-(((n - delay) / width) ** 2))
        budget = gn * (float(e[n + 1]["Ez"][sk, sj, si]) + float(e[n]["Ez"][sk, sj, si]))
        assert abs((W[n + 1] - W[n]) - budget) <= 2e-6 * scale, n
