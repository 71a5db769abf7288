"""Choosing the launch plan and batch size, on the CPU: the library's
candidate set against the candidates the packaged GB300 sweep recorded,
gs_plan_check against the plans that sweep ran and against the rules
gs_set_plan documents, and the pickers' argument checks (which fail before
any CUDA call).  The learned pick itself runs in tests/test_zz_pick_gpu.py."""
import pytest


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300

    return paper_2501_09398_gb300


@pytest.fixture(scope="module")
def tables(g):
    from paper_2501_09398_gb300 import costmodel

    train, held = costmodel.load_tables()
    return costmodel, train + held


def test_candidates_are_the_swept_candidates(g, tables):
    # every one of the 350 swept workloads: the same (plan, S) pairs in the
    # same order as the sweep recorded them
    cm, pairs = tables
    assert len(pairs) == 350
    for w, tab in pairs:
        got = g.gs_candidates(cm._fw(w))
        assert got == [(r["plan"], r["S"]) for r in tab], w


def test_every_swept_plan_passes_the_plan_check(g, tables):
    # all 26,712 swept (plan, S) pairs ran on the GPU (status 0), so the
    # host-side check must accept each plan on its workload
    cm, pairs = tables
    seen = 0
    for w, tab in pairs:
        for plan in {tuple(sorted(r["plan"].items())) for r in tab if r["status"] == 0}:
            g.gs_plan_check(cm._fw(w), dict(plan))
            seen += 1
    assert seen > 3000


@pytest.mark.parametrize("kind,nx,ny,nz,plan,status", [
    ("HEAT3D", 512, 512, 9, dict(kernel=4, temporal_depth=4), "UNSUPPORTED"),  # COLUMN depth 4: 2D or nz <= 8
    ("HEAT3D", 64, 64, 17, dict(kernel=2, temporal_depth=2), "UNSUPPORTED"),   # WAVE needs nz <= 16
    ("HEAT3D", 64, 64, 9, dict(kernel=5), "UNSUPPORTED"),                      # COLUMN_SMEM needs nz <= 8
    ("HEAT2D", 64, 64, 1, dict(kernel=1, temporal_depth=2), "INVALID_ARG"),    # MARCH runs depth 1 only
    ("HEAT2D", 64, 64, 1, dict(kernel=3, temporal_depth=1), "INVALID_ARG"),    # TILE runs depth 2 or 4
    ("HEAT2D", 64, 64, 1, dict(temporal_depth=3), "INVALID_ARG"),
    ("HEAT2D", 64, 64, 1, dict(block_x=48), "INVALID_ARG"),
    ("HEAT2D", 64, 64, 1, dict(block_x=1024), "INVALID_ARG"),                  # thermal block_x <= 512
    ("FDTD3D", 32, 32, 32, dict(temporal_depth=2), "UNSUPPORTED"),
    ("FDTD3D", 32, 32, 32, dict(kernel=2), "INVALID_ARG"),                     # FDTD: COLUMN or MARCH
    ("FDTD3D", 32, 32, 32, dict(block_x=512), "INVALID_ARG"),
    ("HEAT3D", 64, 64, 8, dict(kernel=3, temporal_depth=4, tile_x=256, tile_y=256), "UNSUPPORTED"),  # tile too big
    ("HEAT2D", 64, 64, 2, dict(), "INVALID_ARG"),                              # gs_create refuses the grid
    ("FDTD3D", 32, 32, 31, dict(), "INVALID_ARG"),
    ("FDTD3D", 32, 32, 32, dict(kernel=6, tile_y=-1), "INVALID_ARG"),        # FUSED march: tile_y in [0, 2^20]
    ("FDTD3D", 32, 32, 32, dict(kernel=6, tile_y=(1 << 20) + 1), "INVALID_ARG"),
    ("HEAT2D", 64, 64, 1, dict(kernel=6), "INVALID_ARG"),                      # FUSED is an FDTD kernel
])
def test_plan_check_refuses_what_set_plan_refuses(g, kind, nx, ny, nz, plan, status):
    w = dict(kind=getattr(g, "GS_" + kind), dtype=g.GS_F32, nx=nx, ny=ny, nz=nz)
    with pytest.raises(g.GsError) as e:
        g.gs_plan_check(w, plan)
    assert e.value.status == getattr(g, "GS_ERR_" + status)
    assert "gs_plan_check" in str(e.value)


def test_plan_check_fills_defaults_and_resolves_auto(g):
    w3 = dict(kind=g.GS_HEAT3D, dtype=g.GS_F32, nx=512, ny=512, nz=8)
    p = g.gs_plan_check(w3, {})
    assert (p["kernel"], p["block_x"], p["rows"], p["temporal_depth"]) == (g.GS_KERNEL_COLUMN, 64, 4, 1)
    assert g.gs_plan_check(w3, dict(temporal_depth=2))["kernel"] == g.GS_KERNEL_COLUMN  # nz <= 8: registers
    assert g.gs_plan_check(dict(w3, nz=16), dict(temporal_depth=2))["kernel"] == g.GS_KERNEL_WAVE  # 9..16 planes
    p17 = g.gs_plan_check(dict(w3, nz=17), dict(temporal_depth=2))  # deep stacks at depth 2: planes streamed
    assert (p17["kernel"], p17["block_x"]) == (g.GS_KERNEL_STREAM, 256)
    assert g.gs_plan_check(dict(w3, nz=17), dict(temporal_depth=2, block_x=128))["kernel"] == g.GS_KERNEL_COLUMN  # z-march
    assert g.gs_plan_check(dict(w3, nz=17), dict(temporal_depth=4))["kernel"] == g.GS_KERNEL_TILE
    w2 = dict(kind=g.GS_HEAT2D, dtype=g.GS_BF16, nx=4096, ny=4096, nz=1)
    assert g.gs_plan_check(w2, dict(temporal_depth=4))["kernel"] == g.GS_KERNEL_COLUMN
    assert g.gs_plan_check(w2, {})["rows"] == 8  # large grids: 8 warp rows per block
    wf = dict(kind=g.GS_FDTD3D, dtype=g.GS_F16, nx=128, ny=128, nz=128)
    assert g.gs_plan_check(wf, {})["kernel"] == g.GS_KERNEL_COLUMN
    pf = g.gs_plan_check(wf, dict(kernel=g.GS_KERNEL_FUSED, rows=4, tile_y=8))  # the fused march
    assert (pf["kernel"], pf["rows"], pf["tile_y"]) == (g.GS_KERNEL_FUSED, 4, 8)
    assert g.gs_plan_check(wf, dict(kernel=g.GS_KERNEL_FUSED))["tile_y"] == 0  # its column form


def test_fdtd_candidates_include_the_fused_march(g):
    # FDTD: the fused step's k march (8 planes a block, 4 and 8 rows) among
    # the plans, each with the seven batch sizes; kernels per iteration is 1
    # in its features (2 for the two-launch plans)
    w = dict(kind=g.GS_FDTD3D, dtype=g.GS_F32, nx=256, ny=256, nz=256, n_iters=500)
    cands = g.gs_candidates(w)
    fused = [(p, S) for p, S in cands if p["kernel"] == g.GS_KERNEL_FUSED]
    assert sorted({(p["rows"], p["tile_y"]) for p, _ in fused}) == [(4, 8), (8, 8)]
    assert sorted(S for p, S in fused if p["rows"] == 4) == [0, 1, 10, 50, 100, 500, 1000]
    F = g.gs_features(w, cands)
    for (p, _), f in zip(cands, F):
        assert f[6] == (1.0 if p["kernel"] == g.GS_KERNEL_FUSED else 2.0)
    w2 = dict(kind=g.GS_HEAT2D, dtype=g.GS_F32, nx=512, ny=512, nz=1, n_iters=500)
    assert all(p["kernel"] != g.GS_KERNEL_FUSED and p["tile_y"] == 0 for p, _ in g.gs_candidates(w2))


def test_candidates_argument_checks(g):
    import ctypes

    w = g.gs_workload(g.GS_HEAT2D, g.GS_F32, 64, 64, 1, 100)
    n = ctypes.c_int32()
    assert g._lib.gs_candidates(ctypes.byref(w), None, 0, ctypes.byref(n)) == g.GS_OK
    small = (g.gs_tune_candidate * (n.value - 1))()
    m = ctypes.c_int32()
    assert g._lib.gs_candidates(ctypes.byref(w), small, n.value - 1, ctypes.byref(m)) == g.GS_ERR_INVALID_ARG
    assert m.value == n.value  # the count is reported with the refusal
    ws = g.gs_workload(g.GS_SKELETON, g.GS_F32, 64, 1, 1, 100)
    assert g._lib.gs_candidates(ctypes.byref(ws), None, 0, ctypes.byref(n)) == g.GS_ERR_INVALID_ARG


def test_pickers_refuse_bad_arguments_before_any_cuda_call(g):
    import ctypes

    w = dict(kind=g.GS_HEAT2D, dtype=g.GS_F32, nx=64, ny=64, nz=1, n_iters=100)
    with pytest.raises(g.GsError) as e:
        g.gs_pick([], w)  # no model
    assert e.value.status == g.GS_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    best = g.gs_tune_candidate()
    assert g._lib.gs_pick(arr, 2, ctypes.byref(g._workload(w)), ctypes.byref(best), None) == g.GS_ERR_INVALID_ARG
    S = ctypes.c_int64()
    assert g._lib.gs_pick_analytic(None, 1000, 2, ctypes.byref(S), None) == g.GS_ERR_INVALID_ARG
