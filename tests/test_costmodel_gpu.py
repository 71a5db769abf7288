"""What the learned cost model gains over the method without it.

The network is trained on the GPU by the library's own kernels on the
packaged GB300 sweep (150 workloads) and picks (launch plan, batch size,
temporal depth) for 200 held-out workloads; its regret against each
workload's swept optimum is compared with the paper's analytic picker
(Eqs. 2 and 6 fitted per workload at the default plan) and a fixed S = 100."""
import numpy as np
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
    m, l0, loss = cm.train(X, y)
    try:
        assert loss < 0.01 * l0
        reg = cm.evaluate(m, held)
    finally:
        gs_mlp_destroy(m)
    s = cm.summarize(reg)
    print({k: {q: round(v, 4) for q, v in d.items()} for k, d in s.items()})
    assert s["learned"]["mean"] <= 0.05
    assert s["learned"]["mean"] < 0.5 * s["analytic"]["mean"]
    assert s["learned"]["mean"] < 0.5 * s["fixed_S100"]["mean"]
    assert np.mean(np.array(reg["learned"]) <= np.array(reg["analytic"]) + 1e-12) >= 0.8
