"""Cost-model MLP kernels against the FP64 oracle: loss and gradient,
normalisation, Adam steps (one-step and multi-batch training replayed by the
oracle), convergence on a teacher network, prediction and argmin."""
import numpy as np
import pytest

from oracle import mlp_ref as mr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = (rng.normal(0, 1, (n, mr.NI)) * rng.uniform(0.5, 3, mr.NI) + rng.uniform(-2, 2, mr.NI)).astype(np.float32)
    y = rng.normal(0, 1, n).astype(np.float32)
    return X, y


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_loss_grad_and_normalisation_match_oracle():
    import paper_2501_09398_gb300 as g

    X, y = _data(1000, 40)
    Xd, yd = _dev(X), _dev(y)
    m = g.gs_mlp_create(seed=11)
    try:
        g.gs_mlp_fit_normalization(m, Xd.data_ptr(), X.shape[0])
        mean, inv = g.gs_mlp_get_normalization(m)
        rm, ri = mr.normalization(X.astype(np.float64))
        np.testing.assert_allclose(mean, rm, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(inv, ri, rtol=1e-4)
        p = g.gs_mlp_get_params(m).astype(np.float64)
        loss, grad = g.gs_mlp_loss_grad(m, Xd.data_ptr(), yd.data_ptr(), X.shape[0])
        ref_l = mr.loss(p, X, y, mean.astype(np.float64), inv.astype(np.float64))
        ref_g = mr.grad(p, X, y, mean.astype(np.float64), inv.astype(np.float64))
        assert loss == pytest.approx(ref_l, rel=1e-5)
        assert np.max(np.abs(grad - ref_g)) <= 1e-4 * np.max(np.abs(ref_g)) + 1e-7
    finally:
        g.gs_mlp_destroy(m)


@pytest.mark.parametrize("batch_rows,epochs", [(1000, 1), (300, 2)])
def test_adam_training_matches_oracle_replay(batch_rows, epochs):
    import paper_2501_09398_gb300 as g

    X, y = _data(1000, 41)
    Xd, yd = _dev(X), _dev(y)
    lr = 2e-3
    m = g.gs_mlp_create(seed=12)
    try:
        g.gs_mlp_fit_normalization(m, Xd.data_ptr(), X.shape[0])
        mean, inv = (a.astype(np.float64) for a in g.gs_mlp_get_normalization(m))
        p = g.gs_mlp_get_params(m).astype(np.float64)
        g.gs_mlp_train(m, Xd.data_ptr(), yd.data_ptr(), X.shape[0], epochs, batch_rows, lr)
        got = g.gs_mlp_get_params(m).astype(np.float64)
    finally:
        g.gs_mlp_destroy(m)
    mo, vo, t = np.zeros(mr.NP), np.zeros(mr.NP), 0
    for _ in range(epochs):
        for r0 in range(0, X.shape[0], batch_rows):
            sl = slice(r0, min(r0 + batch_rows, X.shape[0]))
            t += 1
            p, mo, vo = mr.adam_step(p, mr.grad(p, X[sl], y[sl], mean, inv), mo, vo, t, lr)
    assert np.max(np.abs(got - p)) <= 2e-5 * max(1.0, np.max(np.abs(p)))


def test_training_fits_a_teacher_network():
    import paper_2501_09398_gb300 as g

    X, _ = _data(4000, 42)
    rng = np.random.default_rng(5)
    teacher = rng.normal(0, 0.4, mr.NP)
    mean, inv = mr.normalization(X.astype(np.float64))
    y = mr.forward(teacher, X, mean, inv)[0].astype(np.float32)
    Xd, yd = _dev(X), _dev(y)
    m = g.gs_mlp_create(seed=13)
    try:
        g.gs_mlp_fit_normalization(m, Xd.data_ptr(), X.shape[0])
        l0, _ = g.gs_mlp_loss_grad(m, Xd.data_ptr(), yd.data_ptr(), X.shape[0])
        l1 = g.gs_mlp_train(m, Xd.data_ptr(), yd.data_ptr(), X.shape[0], 300, 512, 3e-3)
        assert l1 < 0.05 * l0, (l0, l1)
    finally:
        g.gs_mlp_destroy(m)


def test_predict_and_argmin():
    import torch

    import paper_2501_09398_gb300 as g

    X, _ = _data(3000, 43)
    Xd = _dev(X)
    m = g.gs_mlp_create(seed=14)
    try:
        g.gs_mlp_fit_normalization(m, Xd.data_ptr(), X.shape[0])
        mean, inv = (a.astype(np.float64) for a in g.gs_mlp_get_normalization(m))
        p = g.gs_mlp_get_params(m).astype(np.float64)
        pred = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        g.gs_mlp_predict(m, Xd.data_ptr(), X.shape[0], pred.data_ptr())
        torch.cuda.synchronize()
        got = pred.cpu().numpy().astype(np.float64)
        ref = mr.forward(p, X, mean, inv)[0]
        assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))
        idx, val = g.gs_mlp_argmin(m, Xd.data_ptr(), X.shape[0])
        assert idx == int(np.argmin(got)) and val == pytest.approx(got[idx])
    finally:
        g.gs_mlp_destroy(m)


def test_argmin_ensemble_matches_oracle_mean():
    import paper_2501_09398_gb300 as g

    X, _ = _data(2500, 44)
    Xd, X2d = _dev(X), _dev(X * 2.0 + 1.0)
    models = [g.gs_mlp_create(seed=s) for s in (21, 22, 23)]
    try:
        refs = []
        for i, m in enumerate(models):
            # members standardise with their own statistics
            g.gs_mlp_fit_normalization(m, (X2d if i == 1 else Xd).data_ptr(), X.shape[0])
            mean, inv = (a.astype(np.float64) for a in g.gs_mlp_get_normalization(m))
            refs.append(mr.forward(g.gs_mlp_get_params(m).astype(np.float64), X, mean, inv)[0])
        ref = np.mean(refs, axis=0)
        idx, val = g.gs_mlp_argmin_ensemble(models, Xd.data_ptr(), X.shape[0])
        scale = max(1.0, float(np.max(np.abs(ref))))
        # the pick is a minimum of the oracle mean up to FP32 rounding
        assert ref[idx] <= ref.min() + 1e-5 * scale
        assert abs(val - ref[idx]) <= 1e-5 * scale
        # one member alone is that member's own argmin
        i1, _ = g.gs_mlp_argmin_ensemble(models[:1], Xd.data_ptr(), X.shape[0])
        assert i1 == g.gs_mlp_argmin(models[0], Xd.data_ptr(), X.shape[0])[0]
        with pytest.raises(g.GsError):
            g.gs_mlp_argmin_ensemble([], Xd.data_ptr(), X.shape[0])
    finally:
        for m in models:
            g.gs_mlp_destroy(m)
