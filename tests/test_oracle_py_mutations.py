"""The pins of the oracle's Python parts catch plausible mistakes: each case
plants one mistake in a copy of the oracle package (perf_model.py, the
paper's Eqs. 1-6; mlp_ref.py, the cost model's network, gradient and Adam)
in a temporary directory placed first on the import path of a subprocess,
and runs the matching pin tests there; at least one must fail.  The
unmutated copy passes the same way."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the pins of each file (its checks of the library against the oracle need
# the CUDA package and add nothing here)
PM = ["tests/test_perf_model.py", "-k", "not library"]
MR = ["tests/test_mlp_oracle.py", "-k", "not feature"]

# (name, file, text, replacement, pin tests)
MUTATIONS = [
    ("Eq. 5: a with the wrong sign", "perf_model.py", "return I_k * (T_a - T_i),", "return I_k * (T_i - T_a),", PM),
    ("Eq. 5: b with T_a added", "perf_model.py", "I_k * (T_k + T_i) - T_a + T_l",
     "I_k * (T_k + T_i) + T_a + T_l", PM),
    ("Eq. 3: I launch gaps instead of I - 1", "perf_model.py", "T_a * (I - 1.0)", "T_a * I", PM),
    ("Eq. 6 fitted against S instead of 1/S", "perf_model.py", "np.stack([1.0 / S, np.ones_like(S)], 1), te",
     "np.stack([S, np.ones_like(S)], 1), te", PM),
    ("Eq. 1 maximised", "perf_model.py", "i = int(np.argmin(totals))", "i = int(np.argmax(totals))", PM),
    ("Eq. 2 without the fixed cost", "perf_model.py", "return k_c * np.asarray(S, dtype=np.float64) + b_c",
     "return k_c * np.asarray(S, dtype=np.float64)", PM),
    ("loss gradient without the factor 2", "mlp_ref.py", "dpred = 2.0 * (pred - y) / y.size",
     "dpred = (pred - y) / y.size", MR),
    ("W2 gradient from the pre-activation", "mlp_ref.py", "gW2 = dz2.T @ h1", "gW2 = dz2.T @ z1", MR),
    ("second ReLU left out of the forward pass", "mlp_ref.py", "h2 = np.maximum(z2, 0.0)", "h2 = z2", MR),
    ("Adam without bias correction of m", "mlp_ref.py", "mh = m / (1 - b1 ** t)", "mh = m", MR),
    ("Adam second moment of g, not g^2", "mlp_ref.py", "v = b2 * v + (1 - b2) * g * g", "v = b2 * v + (1 - b2) * g",
     MR),
    ("constant features scaled by 1/0", "mlp_ref.py",
     "inv = np.where(sd > 1e-6, 1.0 / np.where(sd > 0, sd, 1.0), 1.0)",
     "inv = 1.0 / np.where(sd > 0, sd, 1e-300)", MR),
]


def _copy(tmp_path, file=None, old=None, new=None):
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    if file:
        text = (pkg / file).read_text()
        assert text.count(old) == 1, "the mutated text no longer occurs once"
        (pkg / file).write_text(text.replace(old, new))
    return tmp_path


def _run(tmp_path, pins):
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]), OMP_NUM_THREADS="2")
    code = ("import oracle, sys; assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__; "
            "import pytest; sys.exit(pytest.main(sys.argv[2:]))")
    args = [os.path.join(ROOT, p) if p.startswith("tests/") else p for p in pins]
    return subprocess.run([sys.executable, "-c", code, str(tmp_path), *args,
                           "-x", "-q", "-p", "no:cacheprovider", "--rootdir", ROOT],
                          cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name,file,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_pin_fails_on_the_planted_mistake(tmp_path, name, file, old, new, pins):
    r = _run(_copy(tmp_path, file, old, new), pins)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-1500:], r.stderr[-1500:])


@pytest.mark.parametrize("pins", [PM, MR], ids=["perf_model", "mlp_ref"])
def test_the_unmutated_copy_passes(tmp_path, pins):
    r = _run(_copy(tmp_path), pins)
    assert r.returncode == 0, (r.stdout[-1500:], r.stderr[-1500:])
