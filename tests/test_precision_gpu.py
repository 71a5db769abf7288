"""Reduced-precision field storage (bf16 / f16 storage, FP32 arithmetic)
against the FP64 oracle started from the same rounded inputs.

Bars derived from the arithmetic:
* one step: the stored result is the FP32 update rounded to the storage type;
  the FP64 oracle's one-step value rounded to the same type may differ only
  where FP32 and FP64 fall on different sides of a rounding midpoint, i.e. by
  at most one storage ulp, and rarely;
* FDTD over n steps: each leapfrog step rounds every stored value twice (the
  H half-step, then the E half-step), each rounding of relative size <= u
  (unit roundoff 2^-9 bf16, 2^-11 f16), so one step adds an error of norm
  <= 2u times the field's; the scheme is non-dissipative and the roundings
  are unbiased, so they add up like a random walk: relative L2 error
  <= 2 sqrt(n) u;
* thermal over many steps: storage rounding is biased (increments below half
  an ulp are lost, so the field stagnates above its relaxation target) and no
  useful bound exists; the runs must keep the discrete maximum principle, the
  error is printed, and storing theta = T - t_amb (same update with t_amb = 0)
  must cut it.
"""
import math

import numpy as np
import pytest

import gs_inputs
from gsutil import fdtd_concat, fdtd_read, fdtd_setup, fdtd_upload, heat_gpu, max_rel, rel_l2

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {"bf16": 2.0 ** -9, "f16": 2.0 ** -11}
MANT_BITS = {"bf16": 7, "f16": 10}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _ulp(v, dtype):
    a = np.maximum(np.abs(np.asarray(v, dtype=np.float64)), 2.0 ** -14)
    return 2.0 ** (np.floor(np.log2(a)) - MANT_BITS[dtype])


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [(130, 17, 1), (33, 21, 5)])
def test_heat_one_step_rounding(oracle, dtype, shape):
    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=21)
    T0 = gs_inputs.round_to(T0, dtype)
    P = gs_inputs.round_to(P, dtype)
    got = heat_gpu(T0, P, 1, dtype=dtype)
    ref = oracle.heat_run(T0, P, 1, oracle.HEAT_COEFFS_2D if nz == 1 else oracle.HEAT_COEFFS_3D)
    diff = np.abs(got.astype(np.float64) - ref)
    assert np.all(diff <= _ulp(ref, dtype)), float(np.max(diff / _ulp(ref, dtype)))
    near = gs_inputs.round_to(ref.astype(np.float32), dtype)
    assert np.mean(got != near) <= 0.01


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_heat_long_run_properties_and_offset_storage(oracle, dtype):
    nx, ny, n = 256, 128, 1000
    c = oracle.HEAT_COEFFS_2D
    T0, P = gs_inputs.heat_fields(nx, ny, 1, seed=22)
    T0 = gs_inputs.round_to(T0, dtype)
    P = gs_inputs.round_to(P, dtype)
    ref = oracle.heat_run(T0, P, n, c)
    got = heat_gpu(T0, P, n, S=100, dtype=dtype)
    err = max_rel(got, ref)
    # maximum principle: values stay within [t_amb, max T0 + n k max P]
    assert got.min() >= c["t_amb"] - 1e-3 and got.max() <= T0.max() + n * c["k"] * P.max() + 1.0
    # offset storage: theta = T - t_amb, same update with t_amb = 0
    theta0 = gs_inputs.round_to(T0 - np.float32(c["t_amb"]), dtype)
    coeffs = dict(k=c["k"], cx=c["cx"], cy=c["cy"], cz=c["cz"], cz2=c["cz2"], t_amb=0.0)
    th = heat_gpu(theta0, P, n, S=100, dtype=dtype, coeffs=coeffs)
    ref_th = oracle.heat_run(theta0.astype(np.float64) + c["t_amb"], P, n, c)
    err_th = max_rel(th.astype(np.float64) + c["t_amb"], ref_th)
    print(f"{dtype} thermal 1000 steps: max rel err {err:.3e} (T stored), {err_th:.3e} (T - t_amb stored)")
    assert err_th < err


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_fdtd_random_walk_bound(oracle, dtype):
    N, n = 24, 400
    e0 = {k: gs_inputs.round_to(v, dtype) for k, v in gs_inputs.fdtd_random_e(N, seed=23).items()}
    ctx, fields = fdtd_setup(N, dtype)
    import paper_2501_09398_gb300 as g

    try:
        fdtd_upload(ctx, N, e0)
        g.gs_step(ctx, 1, 0)
        one = fdtd_read(ctx, N)
        g.gs_step(ctx, n - 1, 50)
        got = fdtd_read(ctx, N)
    finally:
        g.gs_destroy(ctx)
        del fields
    f = oracle.fdtd_zero_fields(N)
    for k, v in e0.items():
        f[k][...] = v.astype(np.float64)
    oracle.fdtd_run(f, N, 1)
    # H^{1/2} = -s curl E^0 from exactly representable inputs: one rounding
    for k in ("Hx", "Hy", "Hz"):
        assert np.all(np.abs(one[k].astype(np.float64) - f[k]) <= _ulp(f[k], dtype)), k
    oracle.fdtd_run(f, N, n - 1, n0=1)
    err = rel_l2(fdtd_concat(got), fdtd_concat(f))
    bound = 2.0 * math.sqrt(n) * UNIT_ROUNDOFF[dtype]
    print(f"{dtype} FDTD {n} steps: rel L2 {err:.3e} (bound {bound:.3e})")
    assert err <= bound


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_config2_reduced_precision(fdtd_config2_ref, dtype):
    # 128^3 driven cavity, 5000 steps: error reported, bar 2 sqrt(n) u
    N, n, src = 128, 5000, (64, 64, 64)
    ctx, fields = fdtd_setup(N, dtype, src=src)
    import paper_2501_09398_gb300 as g

    try:
        fdtd_upload(ctx, N, {})
        g.gs_step(ctx, n, 100)
        got = fdtd_read(ctx, N)
    finally:
        g.gs_destroy(ctx)
        del fields
    err = rel_l2(fdtd_concat(got), fdtd_concat(fdtd_config2_ref))
    bound = 2.0 * math.sqrt(n) * UNIT_ROUNDOFF[dtype]
    print(f"config2 {dtype} rel L2 {err:.3e} (bound {bound:.3e})")
    assert err <= bound


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [(300, 37, 1), (130, 45, 8), (60, 20, 17), (70, 33, 5)])
def test_temporal_blocking_rounds_every_level(dtype, shape):
    # a depth-t launch rounds each level it computes to the storage type, as
    # t depth-1 launches store (and so round) every step: same bits
    import paper_2501_09398_gb300 as g

    nx, ny, nz = shape
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=41)
    n = 9  # peels n mod t steps at depth 1
    base = heat_gpu(T0, P, n, S=0, dtype=dtype, plan=dict(kernel=g.GS_KERNEL_MARCH, block_x=32, rows=5))
    plans = [dict(kernel=g.GS_KERNEL_TILE, tile_x=16, tile_y=8)]
    if nz <= 16:
        plans.append(dict(kernel=g.GS_KERNEL_WAVE, rows=3, block_x=64))
    if nz <= 8:
        plans.append(dict(kernel=g.GS_KERNEL_COLUMN, block_x=64))
    for depth in (2, 4):
        if nz > 8 and depth == 2:  # deep stacks: the z-marching depth-2 kernel
            got = heat_gpu(T0, P, n, S=4, dtype=dtype, plan=dict(kernel=g.GS_KERNEL_COLUMN, temporal_depth=2, tile_y=7))
            assert np.array_equal(got, base), "z-march"
        for plan in plans:
            got = heat_gpu(T0, P, n, S=4, dtype=dtype, plan=dict(plan, temporal_depth=depth))
            assert np.array_equal(got, base), (depth, plan)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_instance_batch_temporal_depth_reduced_precision(dtype):
    import paper_2501_09398_gb300 as g
    from gsutil import stream_handle

    dims = [(130, 17), (300, 41), (64, 64), (5, 9)]
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=60 + i) for i, (w, h) in enumerate(dims)]
    dt = g.DTYPES[dtype]
    out = []
    for plan in (None, dict(kernel=g.GS_KERNEL_COLUMN, rows=2, temporal_depth=2),
                 dict(kernel=g.GS_KERNEL_COLUMN, rows=4, temporal_depth=4)):
        m = g.gs_multi_create([d[0] for d in dims], [d[1] for d in dims], dt, g.GS_BC_CLAMP, stream_handle())
        bufs = g.MultiFields(m, [d[0] for d in dims], [d[1] for d in dims], dt)
        try:
            if plan:
                g.gs_multi_set_plan(m, **plan)
            for i, (T, P) in enumerate(fields_np):
                g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
                g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
            g.gs_multi_step(m, 11, 5, g.GS_MULTI_FUSED)
            out.append([g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in enumerate(fields_np)])
        finally:
            g.gs_multi_destroy(m)
            del bufs
    for o in out[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(o, out[0]))
