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
* Driven cavity, energy budget: with the soft source added to Ez[src] after
  the E update of step n (E^{n+1} = E~^{n+1} + g(n) e_src), the adjoint
  relation of the two curls gives exactly
  W^{n+1} - W^n = g(n) (Ez^{n+1}[src] + Ez^n[src])
  at every step, so the source-driven run (which has no closed form) is
  pinned step by step: a wrong source time, place, amplitude or sign, or a
  slip in any curl term, breaks it.
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


# ----------------------------------------------------------- media pins --
#
# The lossy-medium Yee update is pinned without restating its coefficients:
# * a table of vacuum rows gives the vacuum scheme bit for bit;
# * in a uniform lossless medium a cavity mode obeys the Yee dispersion with
#   the wave speed 1/sqrt(eps_r mu_r): sin^2 terms scaled by s^2/(eps_r mu_r);
# * in any heterogeneous lossy medium the discrete Poynting theorem holds
#   exactly: with W^n = sum eps |E^n|^2 + sum mu H^{n-1/2} . H^{n+1/2},
#   W^{n+1} - W^n = -(s/2) [ sum sigma (E^{n+1} + E^n)^2
#                            + sum sigma_m H^{n+1/2} (H^{n+3/2} + 2 H^{n+1/2} + H^{n-1/2}) ]
#   (Joule heating of the time-averaged fields), eps, mu, sigma, sigma_m taken
#   at each component's own location; a wrong coefficient, sign, or material
#   lookup breaks it;
# * a swap-symmetric medium keeps the driven field's x <-> y symmetry.

def _per_location(mat, table, q):
    return np.array([row[q] for row in table] + [(1.0, 0.0, 1.0, 0.0)[q]] * (256 - len(table)))[mat]


def test_media_vacuum_table_is_the_vacuum_scheme(oracle):
    N = 10
    mat, _ = gs_inputs.fdtd_media(N, n_mat=3, seed=5)
    f = _fields_from_e(oracle, N, gs_inputs.fdtd_random_e(N, 2))
    g = {k: v.copy() for k, v in f.items()}
    oracle.fdtd_run(f, N, 30, src=(5, 5, 5))
    oracle.fdtd_run(g, N, 30, src=(5, 5, 5), media=(mat, [(1.0, 0.0, 1.0, 0.0)] * 3))
    assert all(np.array_equal(f[c], g[c]) for c in oracle.FDTD_COMPONENTS)


@pytest.mark.parametrize("eps_r,mu_r", [(2.5, 1.5), (6.0, 1.0)])
def test_media_uniform_dielectric_dispersion(oracle, eps_r, mu_r):
    N, s = 16, 0.5
    mode = _mode_field(N, "Ez", 2, 1)
    f = oracle.fdtd_zero_fields(N)
    f["Ez"][...] = mode
    media = (np.ones((N + 1,) * 3, dtype=np.uint8), [(1.0, 0.0, 1.0, 0.0), (eps_r, 0.0, mu_r, 0.0)])
    a = [float(np.sum(f["Ez"] * mode))]
    for _ in range(60):
        oracle.fdtd_run(f, N, 1, courant=s, media=media)
        a.append(float(np.sum(f["Ez"] * mode)))
    cos_pred = 1.0 - 2.0 * s * s / (eps_r * mu_r) * (math.sin(math.pi * 2 / (2 * N)) ** 2
                                                     + math.sin(math.pi * 1 / (2 * N)) ** 2)
    amp = max(abs(v) for v in a)
    checked = 0
    for n in range(1, len(a) - 1):
        if abs(a[n]) > 0.2 * amp:
            assert abs((a[n + 1] + a[n - 1]) / (2.0 * a[n]) - cos_pred) <= 1e-10
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("lossy", [True, False])
def test_media_discrete_poynting_theorem(oracle, lossy):
    N, s = 9, 0.5
    mat, table = gs_inputs.fdtd_media(N, n_mat=4, n_boxes=10, lossy=lossy, seed=11)
    assert len(np.unique(mat)) >= 3
    if lossy:
        assert all(r[1] > 0 and r[3] > 0 for r in table[1:])
    eps, sig, mu, sigm = (_per_location(mat, table, q) for q in range(4))
    E = ("Ex", "Ey", "Ez")
    H = ("Hx", "Hy", "Hz")
    f = _fields_from_e(oracle, N, gs_inputs.fdtd_random_e(N, 4))
    e_hist = [{c: f[c].copy() for c in E}]  # e_hist[n] = E^n
    h_hist = [{c: f[c].copy() for c in H}]  # h_hist[n] = H^{n-1/2}; H^{-1/2} = 0
    for _ in range(40):
        oracle.fdtd_run(f, N, 1, courant=s, media=(mat, table))
        e_hist.append({c: f[c].copy() for c in E})
        h_hist.append({c: f[c].copy() for c in H})

    def W(n):  # sum eps |E^n|^2 + sum mu H^{n-1/2} . H^{n+1/2}
        return (sum(float(np.sum(eps * e_hist[n][c] ** 2)) for c in E)
                + sum(float(np.sum(mu * h_hist[n][c] * h_hist[n + 1][c])) for c in H))

    W0 = W(0)
    assert W0 > 0
    drop = 0.0
    for n in range(0, 38):
        joule = (sum(float(np.sum(sig * (e_hist[n + 1][c] + e_hist[n][c]) ** 2)) for c in E)
                 + sum(float(np.sum(sigm * h_hist[n + 1][c] * (h_hist[n + 2][c] + 2 * h_hist[n + 1][c]
                                                                + h_hist[n][c]))) for c in H))
        assert abs((W(n + 1) - W(n)) + 0.5 * s * joule) <= 1e-12 * W0, n
        drop += W(n) - W(n + 1)
    if lossy:
        assert drop > 1e-4 * W0  # the losses are visible
    else:
        assert abs(drop) <= 1e-12 * W0


def test_media_swap_symmetry(oracle):
    N = 12
    c = N // 2
    mat, table = gs_inputs.fdtd_media(N, n_mat=4, n_boxes=6, seed=8, swap_symmetric=True)
    f = oracle.fdtd_zero_fields(N)
    oracle.fdtd_run(f, N, 90, src=(c, c, c), media=(mat, table))
    Ex, Ey, Ez, Hx, Hy, Hz = (f[k] for k in oracle.FDTD_COMPONENTS)
    scale = np.max(np.abs(Ez))
    sw = lambda a: np.transpose(a, (0, 2, 1))
    tol = 1e-12 * scale
    assert np.max(np.abs(Ez - sw(Ez))) <= tol
    assert np.max(np.abs(Ex - sw(Ey))) <= tol
    assert np.max(np.abs(Hx + sw(Hy))) <= tol
    assert np.max(np.abs(Hz + sw(Hz))) <= tol
    # the medium changes the field: it differs from the vacuum run
    g = oracle.fdtd_zero_fields(N)
    oracle.fdtd_run(g, N, 90, src=(c, c, c))
    assert np.max(np.abs(g["Ez"] - Ez)) > 1e-3 * scale


def test_driven_energy_budget(oracle):
    N, s_c, amp, delay, width = 14, 0.5, 0.7, 30.0, 10.0
    src = (7, 6, 8)
    si, sj, sk = src
    f = oracle.fdtd_zero_fields(N)
    W, ez = [], []
    K = 90
    for n in range(K + 1):
        e_n = {c: f[c].copy() for c in ("Ex", "Ey", "Ez")}
        h_before = {c: f[c].copy() for c in ("Hx", "Hy", "Hz")}
        oracle.fdtd_run(f, N, 1, courant=s_c, n0=n, src=src, amp=amp, delay=delay, width=width)
        W.append(sum(float(np.sum(e_n[c] ** 2)) for c in e_n)
                 + sum(float(np.sum(h_before[c] * f[c])) for c in h_before))
        ez.append(float(e_n["Ez"][sk, sj, si]))
    scale = max(abs(w) for w in W)
    assert scale > 1.0  # the pulse has put energy in
    for n in range(K):
        g = amp * math.exp(-(((n - delay) / width) ** 2))
        assert abs((W[n + 1] - W[n]) - g * (ez[n + 1] + ez[n])) <= 1e-12 * scale, n


def test_driven_media_energy_budget(oracle):
    # The soft source in a lossy dielectric cell, added after the E update.
    # With W^n = sum eps |E^n|^2 + sum mu H^{n-1/2} . H^{n+1/2}, the lossy
    # update and the adjoint curls give, exactly,
    #   W^{n+1} - W^n = -(s/2) [sum sigma (E^{n+1}+E^n)^2
    #                           + sum sigma_m H^{n+1/2}(H^{n+3/2} + 2H^{n+1/2} + H^{n-1/2})]
    #                   + (eps + s sigma / 2)[src] g(n) (Ez^{n+1} + Ez^n)[src]
    # (the source's pre-update value enters the conduction average).  The
    # sigma term at the source tells the order of source and E update apart:
    # in vacuum the two orders agree up to rounding.
    N, s, amp, delay, width = 10, 0.5, 0.7, 12.0, 4.0
    mat, table = gs_inputs.fdtd_media(N, n_mat=4, n_boxes=10, lossy=True, seed=11)
    eps, sig, mu, sigm = (_per_location(mat, table, q) for q in range(4))
    inner = np.argwhere(sig[1:N, 1:N, 1:N] > 0) + 1  # interior Ez unknowns in a lossy cell
    sk, sj, si = (int(v) for v in inner[len(inner) // 2])
    assert sig[sk, sj, si] > 0 and eps[sk, sj, si] > 1
    E, H = ("Ex", "Ey", "Ez"), ("Hx", "Hy", "Hz")
    f = oracle.fdtd_zero_fields(N)
    e_hist = [{c: f[c].copy() for c in E}]
    h_hist = [{c: f[c].copy() for c in H}]
    K = 50
    for n in range(K + 1):
        oracle.fdtd_run(f, N, 1, courant=s, n0=n, src=(si, sj, sk), amp=amp, delay=delay, width=width,
                        media=(mat, table))
        e_hist.append({c: f[c].copy() for c in E})
        h_hist.append({c: f[c].copy() for c in H})

    def W(n):
        return (sum(float(np.sum(eps * e_hist[n][c] ** 2)) for c in E)
                + sum(float(np.sum(mu * h_hist[n][c] * h_hist[n + 1][c])) for c in H))

    scale = max(abs(W(n)) for n in range(K + 1))
    assert scale > 1e-2  # the pulse has put energy in
    src_w = eps[sk, sj, si] + 0.5 * s * sig[sk, sj, si]
    for n in range(K - 1):
        joule = (sum(float(np.sum(sig * (e_hist[n + 1][c] + e_hist[n][c]) ** 2)) for c in E)
                 + sum(float(np.sum(sigm * h_hist[n + 1][c] * (h_hist[n + 2][c] + 2 * h_hist[n + 1][c]
                                                                + h_hist[n][c]))) for c in H))
        g = amp * math.exp(-(((n - delay) / width) ** 2))
        ez = e_hist[n + 1]["Ez"][sk, sj, si] + e_hist[n]["Ez"][sk, sj, si]
        assert abs((W(n + 1) - W(n)) + 0.5 * s * joule - src_w * g * ez) <= 1e-12 * scale, n
