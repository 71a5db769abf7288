"""Pins for the FP64 Yee FDTD oracle (CPU only).

* Discrete energy W^n = sum|E^n|^2 + sum H^{n-1/2} . H^{n+1/2} is exactly
  invariant for the Yee leapfrog in a source-free PEC cavity (the E update
  uses the transpose of the H update's curl); a sign or index slip in any of
  the six curl terms breaks it.
* Cavity modes obey the Yee dispersion relation
  sin(w dt/2) = s sqrt(sin^2(pi m/2N) + sin^2(pi n/2N) + sin^2(pi p/2N)):
  a mode's amplitude a_n satisfies a_{n+1} + a_{n-1} = 2 cos(w dt) a_n.
  One mode per E component exercises every update.
* The soft source: g(delay) = amp and g(delay +- width) = amp/e (width read
  as the 1/e half-width); after one step from rest only Ez[src] = g(0) is
  non-zero.
* With the source at the cavity centre the driven field keeps the cavity's
  mirror and x<->y swap symmetries (E a vector, H a pseudovector).
* Courant number above 1/sqrt(3) is unstable; 0.5 is not.
"""
import math

import numpy as np
import pytest

import gs_inputs


def _fields_from_e(oracle, N, e):
    f = oracle.fdtd_zero_fields(N)
    for c in ("Ex", "Ey", "Ez"):
        f[c][...] = e[c].astype(np.float64)
    return f


def _energy_series(oracle, N, s, n_steps, seed=0):
    f = _fields_from_e(oracle, N, gs_inputs.fdtd_random_e(N, seed))
    e_prev = sum(float(np.sum(f[c] ** 2)) for c in ("Ex", "Ey", "Ez"))  # |E^0|^2
    h_prev = [f[c].copy() for c in ("Hx", "Hy", "Hz")]  # H^{-1/2} = 0
    W = []
    for _ in range(n_steps):
        oracle.fdtd_run(f, N, 1, courant=s)
        h_now = [f[c] for c in ("Hx", "Hy", "Hz")]  # H^{m+1/2}
        W.append(e_prev + sum(float(np.sum(a * b)) for a, b in zip(h_prev, h_now)))
        e_prev = sum(float(np.sum(f[c] ** 2)) for c in ("Ex", "Ey", "Ez"))  # |E^{m+1}|^2
        h_prev = [a.copy() for a in h_now]
    return np.array(W)


def test_energy_invariant_source_free_pec(oracle):
    W = _energy_series(oracle, N=7, s=0.5, n_steps=2000)
    assert np.max(np.abs(W - W[0])) <= 1e-12 * W[0]


def test_unstable_above_courant_limit(oracle):
    N = 6
    f = _fields_from_e(oracle, N, gs_inputs.fdtd_random_e(N, 1))
    e0 = sum(float(np.sum(f[c] ** 2)) for c in ("Ex", "Ey", "Ez"))
    g = {k: v.copy() for k, v in f.items()}
    oracle.fdtd_run(f, N, 400, courant=0.6)
    oracle.fdtd_run(g, N, 400, courant=0.5)
    assert sum(float(np.sum(f[c] ** 2)) for c in ("Ex", "Ey", "Ez")) > 1e6 * e0
    assert sum(float(np.sum(g[c] ** 2)) for c in ("Ex", "Ey", "Ez")) < 10 * e0


def _mode_field(N, comp, m1, m2):
    """Standing mode of one E component, uniform along its own axis."""
    idx = np.arange(N + 1)
    s1 = np.sin(math.pi * m1 * idx / N)
    s2 = np.sin(math.pi * m2 * idx / N)
    a = np.zeros((N + 1,) * 3)
    if comp == "Ez":  # varies in i (m1) and j (m2), k in [0, N)
        a[:N, :, :] = (s2[:, None] * s1[None, :])[None, :, :]
    elif comp == "Ex":  # varies in j (m1) and k (m2), i in [0, N)
        a[:, :, :N] = (s2[:, None] * s1[None, :])[:, :, None]
    else:  # Ey varies in i (m1) and k (m2), j in [0, N)
        a[:, :N, :] = (s2[:, None] * s1[None, :])[:, None, :]
    return a


@pytest.mark.parametrize("comp,m1,m2", [("Ez", 1, 1), ("Ez", 2, 1), ("Ex", 1, 2), ("Ey", 3, 1)])
def test_cavity_mode_dispersion(oracle, comp, m1, m2):
    N, s = 16, 0.5
    mode = _mode_field(N, comp, m1, m2)
    f = oracle.fdtd_zero_fields(N)
    f[comp][...] = mode
    a = [float(np.sum(f[comp] * mode))]
    for _ in range(40):
        oracle.fdtd_run(f, N, 1, courant=s)
        a.append(float(np.sum(f[comp] * mode)))
    cos_pred = 1.0 - 2.0 * s * s * (math.sin(math.pi * m1 / (2 * N)) ** 2 + math.sin(math.pi * m2 / (2 * N)) ** 2)
    amp = max(abs(v) for v in a)
    for n in range(1, len(a) - 1):
        if abs(a[n]) > 0.2 * amp:
            assert abs((a[n + 1] + a[n - 1]) / (2.0 * a[n]) - cos_pred) <= 1e-10
    # the mode stays a mode: nothing leaks into the other E components
    for other in ("Ex", "Ey", "Ez"):
        if other != comp:
            assert np.max(np.abs(f[other])) <= 1e-12


def test_source_reading(oracle):
    assert oracle.fdtd_source(60) == pytest.approx(1.0, rel=0, abs=1e-15)
    assert oracle.fdtd_source(80) == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert oracle.fdtd_source(40) == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert oracle.fdtd_source(0) == pytest.approx(math.exp(-9.0), rel=1e-14)
    N = 8
    f = oracle.fdtd_zero_fields(N)
    oracle.fdtd_run(f, N, 1, src=(4, 4, 4))
    assert f["Ez"][4, 4, 4] == pytest.approx(math.exp(-9.0), rel=1e-14)
    f["Ez"][4, 4, 4] = 0.0
    assert all(np.max(np.abs(v)) == 0.0 for v in f.values())
    # the source sits on Ez[k][j][i] with (i, j, k) = src
    g = oracle.fdtd_zero_fields(N)
    oracle.fdtd_run(g, N, 1, src=(1, 2, 3))
    assert g["Ez"][3, 2, 1] != 0.0 and np.count_nonzero(g["Ez"]) == 1


def test_driven_cavity_symmetries(oracle):
    N = 12
    c = N // 2
    f = oracle.fdtd_zero_fields(N)
    oracle.fdtd_run(f, N, 90, src=(c, c, c))
    Ex, Ey, Ez, Hx, Hy, Hz = (f[k] for k in oracle.FDTD_COMPONENTS)
    scale = np.max(np.abs(Ez))
    assert scale > 0
    tol = 1e-12 * scale
    # x <-> y swap (a reflection): Ex <-> Ey, Ez even; H is a pseudovector
    sw = lambda a: np.transpose(a, (0, 2, 1))  # [k][j][i] -> [k][i][j]
    assert np.max(np.abs(Ez - sw(Ez))) <= tol
    assert np.max(np.abs(Ex - sw(Ey))) <= tol
    assert np.max(np.abs(Hx + sw(Hy))) <= tol
    assert np.max(np.abs(Hz + sw(Hz))) <= tol
    # mirror i -> N - i: Ez on nodes is even; Ex at i+1/2 maps to N-1-i and flips
    assert np.max(np.abs(Ez - Ez[:, :, ::-1])) <= tol
    assert np.max(np.abs(Ex[:, :, :N] + Ex[:, :, N - 1::-1])) <= tol
    # the driven field reached the walls' neighbourhood (the run is not trivial)
    assert np.max(np.abs(Ez[:, :, 1])) > 1e-8 * scale


def test_skeleton_oracle_closed_forms(oracle):
    # the skeleton kernel of Sec. III-C: x <- c x per iteration, so x_n = c^n x_0
    x0 = np.array([1.5, -3.0, 0.25, 7.0])
    assert np.array_equal(oracle.skeleton_run(x0, -1.0, 7), -x0)
    assert np.array_equal(oracle.skeleton_run(x0, 2.0, 10), x0 * 1024.0)
    c = 1.0 + 2.0 ** -8
    np.testing.assert_allclose(oracle.skeleton_run(x0, c, 300), x0 * c ** 300, rtol=1e-13)
