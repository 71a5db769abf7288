"""The paper's performance model (Sec. III-B, Eqs. 1-6): the oracle pinned
to the paper and to algebra, then the library's host-side gs_model_* calls
checked against the oracle (no GPU needed)."""
import math
import os

import numpy as np
import pytest

from oracle import perf_model as pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_fit.txt")


def _table1():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, k_c, b_c, _, a, b, _ = line.split()
        rows[t] = dict(k_c=float(k_c), b_c=float(b_c), a=float(a), b=float(b))
    return rows


def test_eq3_equals_eq6_rearranged():
    # Eq. 5: substituting I = I_k/S into Eq. 3 gives a/S + b exactly.
    rng = np.random.default_rng(1)
    for _ in range(20):
        T_l, T_k, T_i, T_a = rng.uniform(1e-6, 1e-4, 4)
        I_k = int(rng.integers(100, 20000))
        a, b = pm.exec_coeffs(T_l, T_k, T_i, T_a, I_k)
        S = np.array([d for d in pm.divisors(I_k)][:12], dtype=np.float64)
        np.testing.assert_allclose(pm.exec_time_eq3(T_l, T_k, T_i, T_a, S, I_k), pm.exec_time_eq6(a, b, S),
                                   rtol=1e-12)


def test_observation1_sign():
    # Obs. I: batching pays (T_E falls with S) exactly when T_i < T_a, i.e. a > 0.
    a_gain, _ = pm.exec_coeffs(1e-5, 2e-6, 1e-6, 3e-6, 10000)
    a_loss, _ = pm.exec_coeffs(1e-5, 2e-6, 3e-6, 1e-6, 10000)
    assert a_gain > 0 and a_loss < 0
    assert pm.exec_time_eq6(a_gain, 0, 100) < pm.exec_time_eq6(a_gain, 0, 10)


def test_table1_optimum_matches_paper_and_closed_form():
    # Sec. IV-A / Fig. 4: with I_k = 10,000 the optimal iteration batch is
    # around 50-100.  The relaxed minimum of Eq. 1 sits where dT/dS = 0,
    # k_c - a/S^2 = 0, i.e. S* = sqrt(a / k_c).
    t1 = _table1()
    for t, m in t1.items():
        s_star = math.sqrt(m["a"] / m["k_c"])
        best, _ = pm.pick(m, range(1, 2501))
        assert abs(best - s_star) <= 1.0, (t, best, s_star)
    for t in ("1e3", "1e6"):
        best, _ = pm.pick(t1[t], pm.divisors(10000))
        assert 50 <= best <= 100, (t, best)
    # larger workloads gain less (Obs. III): smaller a, so a smaller optimum
    assert math.sqrt(t1["1e7"]["a"] / t1["1e7"]["k_c"]) < math.sqrt(t1["1e3"]["a"] / t1["1e3"]["k_c"])


def test_fit_recovers_exact_model():
    m = dict(k_c=4.2e-6, b_c=1.6e-4, a=1.1e-2, b=2.0e-1)
    S = np.array([1, 2, 5, 10, 50, 100, 500, 1000], dtype=np.float64)
    f = pm.fit(S, pm.creation_time(m["k_c"], m["b_c"], S), pm.exec_time_eq6(m["a"], m["b"], S))
    for k in m:
        assert f[k] == pytest.approx(m[k], rel=1e-9)
    assert f["mae_create"] < 1e-15 and f["mae_exec"] < 1e-12


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300 as lib

    return lib


def test_library_fit_and_pick_match_oracle(g):
    rng = np.random.default_rng(7)
    for trial in range(25):
        m = dict(k_c=rng.uniform(1e-6, 1e-5), b_c=rng.uniform(1e-5, 1e-3), a=rng.uniform(1e-4, 1e-1),
                 b=rng.uniform(1e-3, 1.0))
        S = np.unique(rng.integers(1, 3000, size=int(rng.integers(3, 12)))).astype(np.float64)
        if S.size < 2:
            continue
        tc = pm.creation_time(m["k_c"], m["b_c"], S) * rng.uniform(0.9, 1.1, S.size)
        te = pm.exec_time_eq6(m["a"], m["b"], S) * rng.uniform(0.97, 1.03, S.size)
        ref = pm.fit(S, tc, te)
        got = g.gs_model_fit(S, tc, te)
        for k in ("k_c", "b_c", "a", "b", "mae_create", "mae_exec"):
            assert got[k] == pytest.approx(ref[k], rel=1e-7, abs=1e-15), (trial, k)
        cands = pm.divisors(int(rng.choice([1000, 5000, 10000, 12000])))
        assert g.gs_model_pick(got, cands)[0] == pm.pick(got, cands)[0]
        for s in (1.0, 37.0, 1000.0):
            assert g.gs_model_total(got, s) == pytest.approx(float(pm.total_time(got, s)), rel=1e-12)


def test_library_model_rejects_bad_input(g):
    with pytest.raises(g.GsError):
        g.gs_model_fit([10, 10, 10], [1, 2, 3], [1, 2, 3])
    with pytest.raises(g.GsError):
        g.gs_model_fit([0, 10], [1, 2], [1, 2])
    with pytest.raises(g.GsError):
        g.gs_model_pick(dict(k_c=1, b_c=0, a=1, b=0), [0, 5])
    best, tot = g.gs_model_pick(dict(k_c=1.0, b_c=0.0, a=4.0, b=0.0), [1, 2, 3, 4])
    assert best == 2 and tot == pytest.approx(4.0)
