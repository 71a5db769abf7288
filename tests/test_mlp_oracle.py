"""Pins for the cost model's FP64 oracle (CPU), and the host-side feature
layout of the library (no GPU needed)."""
import math

import numpy as np
import pytest

from oracle import mlp_ref as mr


def _setup(seed=0, n=64):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mr.NP)
    X = rng.normal(0, 1, (n, mr.NI)) * rng.uniform(0.5, 3, mr.NI) + rng.uniform(-2, 2, mr.NI)
    y = rng.normal(0, 1, n)
    mean, inv = mr.normalization(X)
    return p, X, y, mean, inv


def test_grad_matches_central_differences():
    p, X, y, mean, inv = _setup()
    g = mr.grad(p, X, y, mean, inv)
    h = 1e-6
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(mr.NP, 80, replace=False), [mr.NP - 1, 512, 1567, 1600]])
    for i in idx:
        e = np.zeros(mr.NP)
        e[i] = h
        fd = (mr.loss(p + e, X, y, mean, inv) - mr.loss(p - e, X, y, mean, inv)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_normalization_standardises():
    _, X, _, mean, inv = _setup(1, 500)
    Xn = (X - mean) * inv
    np.testing.assert_allclose(Xn.mean(0), 0, atol=1e-12)
    np.testing.assert_allclose(Xn.std(0), 1, rtol=1e-12)
    Xc = X.copy()
    Xc[:, 3] = 7.0
    m2, i2 = mr.normalization(Xc)
    assert m2[3] == 7.0 and i2[3] == 1.0


def test_adam_first_step_closed_form():
    # with m = v = 0, step 1 moves each parameter by lr*g/(|g| + eps)
    rng = np.random.default_rng(2)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = mr.adam_step(p, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300 as lib

    return lib


def test_feature_layout(g):
    w = dict(kind=g.GS_HEAT2D, dtype=g.GS_F32, nx=512, ny=256, nz=1, n_iters=1000)
    f = g.gs_features(w, [(dict(block_x=64, rows=4, temporal_depth=1), 100),
                          (dict(block_x=128, rows=32, temporal_depth=4), 0)])
    # the last two inputs flag the kernel variant: AUTO resolves to COLUMN
    # in 2D, at depth 1 and at depth 4
    expect0 = [9, 8, 0, 1, 0, 0, 1, math.log2(1000), 1, 0, 0, math.log2(100), 0, 6, 2, 1, 1, 0]
    expect1 = [9, 8, 0, 1, 0, 0, 1, math.log2(1000), 1, 0, 0, 0, 1, 7, 5, 4, 1, 0]
    np.testing.assert_allclose(f[0], expect0, rtol=1e-6)
    np.testing.assert_allclose(f[1], expect1, rtol=1e-6)
    w3 = dict(kind=g.GS_FDTD3D, dtype=g.GS_BF16, nx=128, ny=128, nz=128, n_iters=5000)
    f3 = g.gs_features(w3, [(dict(block_x=64, rows=16, temporal_depth=1), 50)])[0]
    assert list(f3[3:7]) == [0, 0, 1, 2] and list(f3[8:11]) == [0, 1, 0] and list(f3[16:]) == [1, 0]
    deep = dict(kind=g.GS_HEAT3D, dtype=g.GS_F32, nx=64, ny=64, nz=16, n_iters=100)
    thin = dict(deep, nz=8)
    one = (dict(block_x=32, rows=16, temporal_depth=1), 10)
    assert list(g.gs_features(deep, [one])[0][16:]) == [1, 0]  # AUTO -> COLUMN (8-plane chunks) above 8 planes
    assert list(g.gs_features(thin, [one])[0][16:]) == [1, 0]
    smem = (dict(block_x=64, rows=4, temporal_depth=1, kernel=g.GS_KERNEL_COLUMN_SMEM), 10)
    march = (dict(block_x=64, rows=4, temporal_depth=1, kernel=g.GS_KERNEL_MARCH), 10)
    assert list(g.gs_features(thin, [smem])[0][16:]) == [1, 1]
    assert list(g.gs_features(thin, [march])[0][16:]) == [0, 0]
    wave = (dict(block_x=64, rows=4, temporal_depth=2), 10)
    assert list(g.gs_features(thin, [wave])[0][16:]) == [0, 0]  # AUTO at depth 2 in 3D -> WAVE
    with pytest.raises(g.GsError):
        g.gs_features(w, [(dict(block_x=0, rows=4, temporal_depth=1), 10)])
