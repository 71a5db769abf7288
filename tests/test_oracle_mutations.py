"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in a copy of oracle.c (on the CPU, in a temporary directory), builds
that copy, and runs the oracle pin tests against it in a subprocess; at
least one pin must fail.  The mistakes are the kind a restatement of the
update could plausibly contain: a dropped or sign-flipped term, swapped
axes, an index off by one, a boundary rule mixed up, the source at the
wrong time or of the wrong shape, a wrong medium coefficient."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_heat.py", "tests/test_oracle_fdtd.py"]

# (name, text in oracle.c, replacement, occurrences replaced: "all" or "first")
MUTATIONS = [
    ("2D: cx and cy swapped",
     "Tn[i] = t + c->k * (P[i] + c->cy * (tn + ts - 2.0 * t)\n                                + c->cx * (te + tw",
     "Tn[i] = t + c->k * (P[i] + c->cx * (tn + ts - 2.0 * t)\n                                + c->cy * (te + tw",
     "all"),
    ("ambient term of the wrong sign", "c->cz * (c->t_amb - t)", "c->cz * (t - c->t_amb)", "all"),
    ("ambient term dropped in 3D", "                                    + c->cz * (c->t_amb - t)\n",
     "\n", "all"),
    ("3D: the power map on every layer", "const double p = (z == 0) ? P[y * nx + x] : 0.0;",
     "const double p = P[y * nx + x];", "all"),
    ("3D: z coupling with a factor 1 instead of 2", "c->cz2 * (tu + td - 2.0 * t)", "c->cz2 * (tu + td - t)", "all"),
    ("3D: upper z-neighbour one row off", "T[i + plane] : 0.0", "T[i + plane - (y > 0 ? nx : 0)] : 0.0", "all"),
    ("Dirichlet-0 reads the centre value", "return bc == OR_BC_CLAMP ? centre : 0.0;", "return centre;", "all"),
    ("clamp reads zero", "return bc == OR_BC_CLAMP ? centre : 0.0;", "return 0.0;", "all"),
    ("odd step counts: last state not copied back", "if (a != T) memcpy", "if (a == T && a != T) memcpy", "all"),
    ("Hx updated with the wrong sign", "Hx[c] -= s *", "Hx[c] += s *", "all"),
    ("Hy curl with a forward difference in the wrong direction",
     "Hy[c] -= s * ((Ex[yee(N, i, j, k + 1)] - Ex[c])", "Hy[c] -= s * ((Ex[c] - Ex[yee(N, i, j, k + 1)])", "all"),
    ("Ez backward difference reads the wrong neighbour",
     "Ez[c] += s * ((Hy[c] - Hy[yee(N, i - 1, j, k)])", "Ez[c] += s * ((Hy[c] - Hy[yee(N, i, j - 1, k)])", "all"),
    ("Ex written on the PEC walls y = 0", "if (i < N && j >= 1 && j <= N - 1 && k >= 1 && k <= N - 1) /* Ex */",
     "if (i < N && j >= 0 && j <= N - 1 && k >= 1 && k <= N - 1) /* Ex */", "all"),
    ("source one step late", "+= or_fdtd_source((double)n, amp", "+= or_fdtd_source((double)(n + 1), amp", "first"),
    ("source added before the E update",
     "        or_fdtd_e(N, s, Ex, Ey, Ez, Hx, Hy, Hz);\n        if (src_on)\n"
     "            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n",
     "        if (src_on)\n            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n"
     "        or_fdtd_e(N, s, Ex, Ey, Ez, Hx, Hy, Hz);\n", "all"),
    ("media: source added before the E update",
     "        or_fdtd_e_media(N, tab, mat, Ex, Ey, Ez, Hx, Hy, Hz);\n        if (src_on)\n"
     "            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n",
     "        if (src_on)\n            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n"
     "        or_fdtd_e_media(N, tab, mat, Ex, Ey, Ez, Hx, Hy, Hz);\n", "all"),
    ("source added before the E update in both runs",
     ("        or_fdtd_e(N, s, Ex, Ey, Ez, Hx, Hy, Hz);\n        if (src_on)\n"
      "            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n",
      "        or_fdtd_e_media(N, tab, mat, Ex, Ey, Ez, Hx, Hy, Hz);\n        if (src_on)\n"
      "            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n"),
     ("        if (src_on)\n            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n"
      "        or_fdtd_e(N, s, Ex, Ey, Ez, Hx, Hy, Hz);\n",
      "        if (src_on)\n            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);\n"
      "        or_fdtd_e_media(N, tab, mat, Ex, Ey, Ez, Hx, Hy, Hz);\n"), "all"),
    ("source width read as sigma", "return amp * exp(-u * u);", "return amp * exp(-u * u / 2.0);", "all"),
    ("media: conduction not averaged over the two time levels", "const double ae = sigma * s / (2.0 * eps_r);",
     "const double ae = sigma * s / eps_r;", "all"),
    ("media: magnetic loss ignored", "const double ah = sigma_m * s / (2.0 * mu_r);", "const double ah = 0.0;",
     "all"),
    ("media: E takes the material of the cell below in x",
     "                const or_medium m = tab[mat[c]];\n                if (i < N && j >= 1",
     "                const or_medium m = tab[mat[i > 0 ? c - 1 : c]];\n                if (i < N && j >= 1", "all"),
]


def _mutant(tmp_path, old, new, which):
    with open(SRC) as f:
        text = f.read()
    pairs = list(zip(old, new)) if isinstance(old, tuple) else [(old, new)]
    for o, n in pairs:
        assert text.count(o) >= 1, "the mutated text no longer occurs in oracle.c"
        text = text.replace(o, n) if which == "all" else text.replace(o, n, 1)
    d = tmp_path / "oracle"
    d.mkdir()
    (d / "oracle.c").write_text(text)
    return str(d / "oracle.c")


@pytest.mark.parametrize("name,old,new,which", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_pin_fails_on_the_planted_mistake(tmp_path, name, old, new, which):
    src = _mutant(tmp_path, old, new, which)
    env = dict(os.environ, GS_ORACLE_SRC=src, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert "failed" in r.stdout.splitlines()[-1] if r.stdout else False, (name, r.stdout[-800:], r.stderr[-800:])
    assert r.returncode == 1, (name, r.returncode, r.stdout[-800:])


def test_the_unmutated_copy_passes(tmp_path):
    # the harness itself: the same copy-and-build route with no mistake passes
    src = _mutant(tmp_path, "double or_fdtd_source", "double or_fdtd_source", "all")
    env = dict(os.environ, GS_ORACLE_SRC=src, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-800:]
