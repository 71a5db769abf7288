"""The packaged GB300 sweep and the pickers that need no GPU (the paper's
analytic model, a fixed S), checked on CPU."""
import math

import pytest


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__

    __graft_entry__._builder().build()
    from paper_2501_09398_gb300 import costmodel

    return costmodel


def test_packaged_sweep_is_complete(cm):
    train, held = cm.load_tables()
    assert len(train) == 150 and len(held) == 200
    for w, tab in train + held:
        assert len(tab) == len(cm.candidates(w))
        ok = [r for r in tab if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
        assert len(ok) >= len(tab) // 2
        assert all(r["ms_per_iter"] > 0 for r in ok)
    # the held-out workloads are the seed-4242 draw
    assert [w for w, _ in held[:5]] == cm.sample_workloads(200, seed=4242)[:5]


def test_analytic_and_fixed_pickers_run_on_the_sweep(cm):
    _, held = cm.load_tables()
    for w, tab in held[:40]:
        ra = cm.regret(w, tab, cm.pick_analytic(w, tab))
        rf = cm.regret(w, tab, cm.pick_fixed(w, tab))
        assert ra >= 0 and rf >= 0


def test_calibration_cost_of_the_analytic_picker(cm):
    # the analytic picker must time every batch size it fits Eqs. 2/6 to:
    # at least one build and one launch each, i.e. the sum over the default
    # plan's swept rows of T_C + S * t_iter; charging it can only add regret
    _, held = cm.load_tables()
    for w, tab in held[:40]:
        dp = cm.default_plan(w)
        rows = [r for r in tab if r["plan"] == dp and r["S"] > 0 and r["status"] == 0]
        assert len(rows) >= 2
        expect = sum(r["build_seconds"] * 1e3 + r["S"] * r["ms_per_iter"] for r in rows)
        assert math.isclose(cm.calibration_ms(w, tab), expect, rel_tol=1e-12)
        assert cm.calibration_ms(w, tab) > 0
        # the iterations alone exceed 1 + 10 + 50 + 100 + 500 + 1000 of the fastest plan's
        fastest = min(r["ms_per_iter"] for r in tab if r["status"] == 0 and math.isfinite(r["ms_per_iter"]))
        assert cm.calibration_ms(w, tab) >= 1661 * fastest * (1 - 1e-9)
