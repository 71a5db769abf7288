"""What the learned cost model gains over the method without it.

The network is trained on the GPU by the library's own kernels on the
packaged GB300 sweep (150 workloads) and picks (launch plan, batch size,
temporal depth) for 200 held-out workloads without running them; its
regret against each workload's swept optimum is compared with a fixed
S = 100 and with the paper's analytic picker (Eqs. 2 and 6 fitted per
workload at the default plan, depth 1: it cannot choose a plan or a
temporal depth).  The analytic picker also needs the workload's own build
and run times at six batch sizes; it is reported with that calibration free
and with the least of it charged (one build and one launch per batch
size)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def test_learned_picker_within_5pct_and_beats_analytic():
    from paper_2501_09398_gb300 import costmodel as cm
    from paper_2501_09398_gb300 import gs_mlp_destroy

    train, held = cm.load_tables()
    X, y = cm.training_set(train)
    models, l0, loss = cm.train(X, y)
    try:
        assert all(b < 0.01 * a for a, b in zip(l0, loss))
        reg = cm.evaluate(models, held)
    finally:
        for m in models:
            gs_mlp_destroy(m)
    s = cm.summarize(reg)
    print({k: {q: round(v, 4) for q, v in d.items()} for k, d in s.items()})
    assert s["learned"]["mean"] <= 0.05
    assert s["learned"]["mean"] < 0.5 * s["fixed_S100"]["mean"]
    assert s["learned"]["p95"] < 0.5 * s["fixed_S100"]["p95"]
    # the analytic model picks S at the default plan (depth 1) and cannot
    # choose a plan or temporal depth: its misses are large where another
    # wins, so even with its calibration free the learned picks halve its
    # mean and its tail
    assert s["learned"]["mean"] < 0.5 * s["analytic"]["mean"]
    assert s["learned"]["p95"] < 0.5 * s["analytic"]["p95"]
    # and it needs measurements of each new workload: charged for them it
    # loses by far to the pick that needs none
    assert s["learned"]["mean"] < 0.1 * s["analytic_with_calibration"]["mean"]
