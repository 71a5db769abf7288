"""FDTD in lossy heterogeneous media on the GPU against the FP64 oracle.

A material map (uint8 ids, one per component location) and a table of
(eps_r, sigma, mu_r, sigma_m) rows drive the lossy-medium Yee update in the
column kernels and in the fused step's k march.  Checked: parity with the
oracle (relative L2 <= 1e-4, the
FDTD bar) on ragged cube sizes with the driven source and from a random
field, bit-identity of graph batches and the device loop with per-step
launches, a vacuum table reproducing the vacuum kernels bit for bit, the
discrete Poynting theorem on the GPU's own fields, reduced-precision
storage within the random-walk bar 2 sqrt(n) u, and the error paths."""
import math

import numpy as np
import pytest

import gs_inputs
from gsutil import FDTD_NAMES, FDTD_RL2, fdtd_concat, fdtd_read, fdtd_setup, fdtd_upload, rel_l2

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _gpu(N, n, S=0, media=None, src=None, init=None, plan=None, dtype="f32"):
    import paper_2501_09398_gb300 as g

    ctx, fields = fdtd_setup(N, dtype, plan=plan, src=src, media=media)
    try:
        fdtd_upload(ctx, N, init or {})
        g.gs_step(ctx, n, S)
        return fdtd_read(ctx, N)
    finally:
        g.gs_destroy(ctx)
        del fields


def _ref(oracle, N, n, media, src=None, init=None):
    f = oracle.fdtd_zero_fields(N)
    for k, v in (init or {}).items():
        f[k][...] = np.asarray(v, dtype=np.float64)
    return oracle.fdtd_run(f, N, n, courant=0.5, src=src, media=media)


@pytest.mark.parametrize("N", [11, 20, 37])
def test_driven_media_parity(oracle, N):
    media = gs_inputs.fdtd_media(N, n_mat=5, n_boxes=9, seed=N)
    c = N // 2
    n = 200
    ref = _ref(oracle, N, n, media, src=(c, c, c))
    got = _gpu(N, n, media=media, src=(c, c, c))
    err = rel_l2(fdtd_concat(got), fdtd_concat(ref))
    assert err <= FDTD_RL2, err
    # the medium matters: the vacuum field is far from this one
    vac = _ref(oracle, N, n, None, src=(c, c, c))
    assert rel_l2(fdtd_concat(vac), fdtd_concat(ref)) > 100 * FDTD_RL2


def test_random_field_media_parity(oracle):
    N, n = 24, 300
    media = gs_inputs.fdtd_media(N, n_mat=4, seed=3)
    e0 = gs_inputs.fdtd_random_e(N, seed=31)
    ref = _ref(oracle, N, n, media, init=e0)
    got = _gpu(N, n, media=media, init=e0)
    assert rel_l2(fdtd_concat(got), fdtd_concat(ref)) <= FDTD_RL2


def test_media_aligned_grid_parity(oracle):
    # N = 128: the aligned layout (lane 31 takes the i = N column) with the
    # media coefficients, from random values in every entry, source on the
    # i = N wall
    N, n = 128, 10
    media = gs_inputs.fdtd_media(N, n_mat=6, n_boxes=12, seed=5)
    init = gs_inputs.fdtd_random_all(N, seed=6)
    src = (N, 40, 70)
    ref = _ref(oracle, N, n, media, src=src, init=init)
    got = _gpu(N, n, 4, media=media, src=src, init=init)
    assert rel_l2(fdtd_concat(got), fdtd_concat(ref)) <= FDTD_RL2
    wall = got["Hx"][:, :, N].astype(np.float64)
    assert np.linalg.norm(wall - ref["Hx"][:, :, N]) <= FDTD_RL2 * np.linalg.norm(ref["Hx"][:, :, N])


def test_media_graphs_bit_identical():
    N, n = 21, 45
    media = gs_inputs.fdtd_media(N, n_mat=4, seed=9)
    src = (7, 11, 5)
    base = _gpu(N, n, 0, media=media, src=src)
    for S, plan in ((1, None), (7, None), (45, None), (9, dict(use_pdl=1)), (9, dict(rows=1)), (9, dict(rows=8)),
                    (6, dict(graph_loop=1))):
        got = _gpu(N, n, S, media=media, src=src, plan=plan)
        assert all(np.array_equal(got[k], base[k]) for k in FDTD_NAMES), (S, plan)


@pytest.mark.parametrize("N,src", [(21, (7, 11, 5)), (128, (128, 40, 70)), (256, (128, 100, 60))])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_media_fused_march_bit_identical(N, src, dtype):
    # the fused step marching in k with the media coefficients (per-cell
    # ids, the table's H and E rows in shared memory) against the two-launch
    # column kernels, from random values in every entry: ragged, aligned,
    # and aligned with two blocks along i
    import paper_2501_09398_gb300 as g

    media = gs_inputs.fdtd_media(N, n_mat=6, n_boxes=12, seed=N)
    init = gs_inputs.fdtd_random_all(N, seed=N + 3)
    n = 7
    base = _gpu(N, n, 0, media=media, src=src, init=init, dtype=dtype)
    for S, plan in ((0, dict(rows=4, tile_y=1)), (3, dict(rows=2, tile_y=5)), (7, dict(rows=8, tile_y=300))):
        got = _gpu(N, n, S, media=media, src=src, init=init, dtype=dtype,
                   plan=dict(kernel=g.GS_KERNEL_FUSED, **plan))
        assert all(np.array_equal(got[k], base[k]) for k in FDTD_NAMES), (S, plan)


def test_vacuum_table_is_the_vacuum_kernel():
    N, n = 19, 60
    mat, _ = gs_inputs.fdtd_media(N, n_mat=3, seed=4)
    vac = _gpu(N, n, 10, src=(9, 9, 9))
    got = _gpu(N, n, 10, media=(mat, [(1.0, 0.0, 1.0, 0.0)] * 3), src=(9, 9, 9))
    assert all(np.array_equal(got[k], vac[k]) for k in FDTD_NAMES)


def test_poynting_theorem_on_gpu_fields():
    # W^{n+1} - W^n = -(s/2) [sum sigma (E^{n+1}+E^n)^2
    #                         + sum sigma_m H^{n+1/2}(H^{n+3/2} + 2H^{n+1/2} + H^{n-1/2})]
    # on the GPU's own FP32 fields, one step at a time from a random E
    import paper_2501_09398_gb300 as g

    N, s = 16, 0.5
    mat, table = gs_inputs.fdtd_media(N, n_mat=4, seed=12)
    per = [np.array([r[q] for r in table] + [(1.0, 0.0, 1.0, 0.0)[q]] * (256 - len(table)))[mat] for q in range(4)]
    eps, sig, mu, sigm = per
    ctx, fields = fdtd_setup(N, media=(mat, table))
    E, H = ("Ex", "Ey", "Ez"), ("Hx", "Hy", "Hz")
    try:
        fdtd_upload(ctx, N, gs_inputs.fdtd_random_e(N, seed=5))
        hist = [fdtd_read(ctx, N)]
        for _ in range(12):
            g.gs_step(ctx, 1, 0)
            hist.append(fdtd_read(ctx, N))
    finally:
        g.gs_destroy(ctx)
        del fields
    h = [{c: np.zeros_like(hist[0][c], dtype=np.float64) for c in H}] + [
        {c: f[c].astype(np.float64) for c in H} for f in hist[1:]]  # h[n] = H^{n-1/2}
    e = [{c: f[c].astype(np.float64) for c in E} for f in hist]

    def W(n):
        return (sum(float(np.sum(eps * e[n][c] ** 2)) for c in E)
                + sum(float(np.sum(mu * h[n][c] * h[n + 1][c])) for c in H))

    W0 = W(0)
    for n in range(10):
        joule = (sum(float(np.sum(sig * (e[n + 1][c] + e[n][c]) ** 2)) for c in E)
                 + sum(float(np.sum(sigm * h[n + 1][c] * (h[n + 2][c] + 2 * h[n + 1][c] + h[n][c]))) for c in H))
        assert abs(W(n + 1) - W(n) + 0.5 * s * joule) <= 2e-6 * W0, n


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_media_reduced_precision_bound(oracle, dtype):
    N, n = 24, 400
    media = gs_inputs.fdtd_media(N, n_mat=4, seed=6)
    e0 = {k: gs_inputs.round_to(v, dtype) for k, v in gs_inputs.fdtd_random_e(N, seed=24).items()}
    got = _gpu(N, n, 50, media=media, init=e0, dtype=dtype)
    ref = _ref(oracle, N, n, media, init=e0)
    err = rel_l2(fdtd_concat(got), fdtd_concat(ref))
    bound = 2.0 * math.sqrt(n) * UNIT_ROUNDOFF[dtype]
    print(f"{dtype} FDTD media {n} steps: rel L2 {err:.3e} (bound {bound:.3e})")
    assert err <= bound


def test_media_error_paths():
    import paper_2501_09398_gb300 as g

    N = 8
    ctx, fields = fdtd_setup(N)
    try:
        fdtd_upload(ctx, N, {})
        g.gs_set_fdtd_media(ctx, [(2.0, 0.0, 1.0, 0.0)])
        with pytest.raises(g.GsError) as e:  # no material map bound
            g.gs_step(ctx, 1, 0)
        assert e.value.status == g.GS_ERR_STATE
        for bad, status in (((0.0, 0.0, 1.0, 0.0), g.GS_ERR_INVALID_ARG), ((1.0, -1.0, 1.0, 0.0), g.GS_ERR_INVALID_ARG),
                            ((float("nan"), 0.0, 1.0, 0.0), g.GS_ERR_NUMERIC)):
            with pytest.raises(g.GsError) as e:
                g.gs_set_fdtd_media(ctx, [bad])
            assert e.value.status == status
        with pytest.raises(g.GsError) as e:
            g.gs_set_fdtd_media(ctx, [(1.0, 0.0, 1.0, 0.0)] * 257)
        assert e.value.status == g.GS_ERR_INVALID_ARG
        g.gs_set_fdtd_media(ctx, [])  # back to vacuum: steps without a map
        g.gs_step(ctx, 2, 0)
    finally:
        g.gs_destroy(ctx)
        del fields
    media = gs_inputs.fdtd_media(N, n_mat=2, seed=1)
    ctx, fields = fdtd_setup(N, media=media, plan=dict(kernel=g.GS_KERNEL_MARCH))
    try:
        with pytest.raises(g.GsError) as e:
            g.gs_step(ctx, 1, 0)
        assert e.value.status == g.GS_ERR_UNSUPPORTED
        with pytest.raises(g.GsError):
            g.gs_upload(ctx, g.GS_FIELD_MAT, np.zeros((N + 1) ** 3, dtype=np.float32))
    finally:
        g.gs_destroy(ctx)
        del fields
