"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a copy
of oracle.c built with -fsanitize=address,undefined (in a temporary
directory, loaded in a subprocess with the ASan runtime preloaded) passes
every oracle pin test with no sanitizer report, and the same harness reports
a read one row past a field's end planted in another copy, so a clean run
means the oracle's index arithmetic stays in its arrays."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_heat.py", "tests/test_oracle_fdtd.py"]
FLAGS = "-fsanitize=address,undefined -fno-omit-frame-pointer -fno-sanitize-recover=undefined -g"


def _runtime():
    path = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not path or not os.path.isabs(path) or not os.path.exists(path):
        pytest.skip("no AddressSanitizer runtime for gcc")
    return path


def _run(tmp_path, text):
    d = tmp_path / "oracle"
    d.mkdir()
    (d / "oracle.c").write_text(text)
    env = dict(os.environ, GS_ORACLE_SRC=str(d / "oracle.c"), GS_ORACLE_CFLAGS=FLAGS, LD_PRELOAD=_runtime(),
               ASAN_OPTIONS="detect_leaks=0", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-s", "-p", "no:cacheprovider"], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=900)


def test_oracle_pins_pass_clean_under_asan_and_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    with open(SRC) as f:
        r = _run(tmp_path, f.read())
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-2000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-2000:]


def test_the_harness_reports_a_read_past_the_end(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    with open(SRC) as f:
        text = f.read()
    old = "const double ts = nb(y < ny - 1, y < ny - 1 ? T[i + nx] : 0.0, t, bc);"
    assert text.count(old) == 2
    # the 2D step reads the row below even on the last row
    text = text.replace(old, "const double ts = nb(y < ny - 1, T[i + nx], t, bc);", 1)
    r = _run(tmp_path, text)
    assert r.returncode != 0
    assert "AddressSanitizer" in r.stdout + r.stderr
