"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer.

A copy of libgraphstep is compiled from csrc/ with -fsanitize=address and
-fsanitize=undefined on the host side (into a temporary directory; the
in-tree library is untouched) and loaded with ctypes in a subprocess that
preloads the ASan runtime and allocates through malloc.  That process drives
every entry point that runs without a GPU: the candidate set and the plan
check over all 350 swept workloads of the packaged GB300 sweep, the feature
rows of every candidate, the paper's model fit and pick, the pitch rule, the
status strings, and the argument checks of gs_create, gs_multi_create and
gs_multi_step_noalloc.  It must finish with no sanitizer report; a planted
write one feature row past a buffer's end must be reported."""
import ctypes
import glob
import importlib.util
import os
import subprocess
import sys
import concurrent.futures as cf

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined", "-Xcompiler",
       "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=undefined"]

# The structs the harness uses, as the binding declares them (checked below).
STRUCTS = '''
import ctypes
i32, i64 = ctypes.c_int32, ctypes.c_int64
class gs_plan(ctypes.Structure):
    _fields_ = [(n, i32) for n in ("block_x", "rows", "tile_x", "tile_y", "temporal_depth", "use_pdl",
                                   "device_launch", "kernel", "graph_loop", "traverse")]
class gs_tune_candidate(ctypes.Structure):
    _fields_ = [("plan", gs_plan), ("batch_size", i64)]
class gs_workload(ctypes.Structure):
    _fields_ = [("kind", i32), ("dtype", i32), ("nx", i64), ("ny", i64), ("nz", i64), ("n_iters", i64)]
class gs_model(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("k_c", "b_c", "a", "b", "mae_create", "mae_exec")]
class gs_instance(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_void_p), ("T1", ctypes.c_void_p), ("P", ctypes.c_void_p), ("nx", i64),
                ("ny", i64), ("pitch", i64), ("p_pitch", i64)]
class gs_heat_coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("k", "cx", "cy", "cz", "cz2", "t_amb")]
'''

DRIVER = STRUCTS + '''
import gzip, json, math, random, sys
lib = ctypes.CDLL(sys.argv[1])
KIND = {"heat2d": 0, "heat3d": 1, "fdtd": 2}
with gzip.open(sys.argv[2], "rt") as f:
    d = json.load(f)
pairs = d["train"] + d["heldout"]
P = ctypes.POINTER
fp = P(ctypes.c_float)
n_checked = 0
for w, tab in pairs:
    wl = gs_workload(KIND[w["kind"]], w["dtype"], w["nx"], w["ny"], w["nz"], w["n_iters"])
    n = i32()
    assert lib.gs_candidates(ctypes.byref(wl), None, 0, ctypes.byref(n)) == 0
    arr = (gs_tune_candidate * n.value)()
    assert lib.gs_candidates(ctypes.byref(wl), arr, n.value, ctypes.byref(n)) == 0
    short = (gs_tune_candidate * (n.value - 1))()
    assert lib.gs_candidates(ctypes.byref(wl), short, n.value - 1, ctypes.byref(n)) != 0
    for c in arr:
        out = gs_plan()
        assert lib.gs_plan_check(ctypes.byref(wl), ctypes.byref(c.plan), ctypes.byref(out)) == 0
        n_checked += 1
    rows = (ctypes.c_float * (len(arr) * 18 - (18 if sys.argv[3] == "overflow" else 0)))()
    assert lib.gs_features(ctypes.byref(wl), arr, len(arr), ctypes.cast(rows, fp)) == 0
# plans the check refuses, and grids gs_create refuses
bad = gs_plan(48, 4, 0, 0, 1, 0, 0, 0, 0, 0)
wl = gs_workload(0, 0, 64, 64, 1, 100)
assert lib.gs_plan_check(ctypes.byref(wl), ctypes.byref(bad), None) != 0
wl = gs_workload(0, 0, 64, 64, 2, 100)
assert lib.gs_plan_check(ctypes.byref(wl), ctypes.byref(gs_plan()), None) != 0
h = ctypes.c_void_p()
for args in ((7, 8, 8, 1, 0, 0), (0, 0, 8, 1, 0, 0), (2, 8, 8, 9, 0, 2), (0, 8, 8, 1, 9, 0), (0, 8, 8, 1, 0, 2)):
    assert lib.gs_create(ctypes.byref(h), *args, None) != 0
# the paper's model
rng = random.Random(1)
S = [1.0, 10.0, 50.0, 100.0, 500.0, 1000.0]
D = ctypes.c_double * 6
m = gs_model()
assert lib.gs_model_fit(D(*S), D(*[1e-6 * s + 3e-5 + rng.uniform(0, 1e-7) for s in S]),
                        D(*[2e-2 / s + 1e-2 for s in S]), 6, ctypes.byref(m)) == 0
best, tot = i64(), ctypes.c_double()
assert lib.gs_model_pick(ctypes.byref(m), (i64 * 6)(*[int(s) for s in S]), 6, ctypes.byref(best), ctypes.byref(tot)) == 0
assert lib.gs_model_total(ctypes.byref(m), ctypes.c_double(100.0), ctypes.byref(tot)) == 0
assert lib.gs_model_fit(D(*S), D(*S), D(*S), 1, ctypes.byref(m)) != 0
# pitch rule, status strings, messages
p = i64()
for dt in (0, 1, 2):
    for width in (1, 7, 8, 129, 4096):
        assert lib.gs_required_pitch(dt, width, ctypes.byref(p)) == 0 and p.value >= width
lib.gs_status_string.restype = ctypes.c_char_p
for s in range(-1, 10):
    assert lib.gs_status_string(s)
lib.gs_last_error.restype = ctypes.c_char_p
assert lib.gs_last_error(None) is not None
# argument checks of the batch calls (each case invalid, nothing reaches a device)
ny = (i64 * 2)(64, 0)
assert lib.gs_multi_create(ctypes.byref(h), 2, (i64 * 2)(64, 32), ny, 0, 0, None) != 0
inst = (gs_instance * 2)(gs_instance(0x10000, 0x11000, 0x12000, 64, 32, 64, 64),
                         gs_instance(0x10000, 0x11000, 0x12004, 64, 32, 64, 64))
c = gs_heat_coeffs(0.5, 0.1, 0.1, 0.01, 0.05, 80.0)
assert lib.gs_multi_step_noalloc(inst, 2, 0, i64(10), ctypes.byref(c), 0, 0, None, None) != 0
assert lib.gs_multi_step_noalloc(inst, 300, 0, i64(10), ctypes.byref(c), 0, 0, None, None) != 0
print("checked", n_checked)
'''


@pytest.fixture(scope="module")
def sanitized_lib(tmp_path_factory):
    runtime = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(runtime) or not os.path.exists(runtime):
        pytest.skip("no AddressSanitizer runtime for gcc")
    spec = importlib.util.spec_from_file_location("_gs_build_san", os.path.join(ROOT, "paper_2501_09398_gb300",
                                                                                 "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    out = tmp_path_factory.mktemp("asan")
    srcs = sorted(glob.glob(os.path.join(b.CSRC, "*.cu")))

    def comp(src):
        obj = str(out / (os.path.basename(src)[:-3] + ".o"))
        r = subprocess.run([b.nvcc(), "-c", src, "-o", obj] + b.NVCC_FLAGS + SAN, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(comp, srcs))
    lib = str(out / "libgraphstep_san.so")
    r = subprocess.run([b.nvcc(), "-shared", "-o", lib] + objs + b.ARCH + ["-Xcompiler", "-fPIC", "-cudart", "static"]
                       + SAN, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return lib, runtime, out


def _drive(sanitized_lib, mode):
    lib, runtime, out = sanitized_lib
    script = out / "driver.py"
    script.write_text(DRIVER)
    data = os.path.join(ROOT, "paper_2501_09398_gb300", "data", "costmodel_sweep_gb300.json.gz")
    env = dict(os.environ, LD_PRELOAD=runtime, PYTHONMALLOC="malloc", ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    return subprocess.run([sys.executable, str(script), lib, data, mode], env=env, capture_output=True, text=True,
                          timeout=600)


def test_driver_structs_are_the_bindings():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300 as g

    ns = {}
    exec(STRUCTS, ns)
    for name in ("gs_plan", "gs_tune_candidate", "gs_workload", "gs_model", "gs_instance", "gs_heat_coeffs"):
        mine, theirs = ns[name], getattr(g, name)
        assert [f for f, _ in mine._fields_] == [f for f, _ in theirs._fields_], name
        assert ctypes.sizeof(mine) == ctypes.sizeof(theirs), name
        for f, _ in mine._fields_:
            assert getattr(mine, f).offset == getattr(theirs, f).offset, (name, f)


def test_host_code_is_clean_under_asan_and_ubsan(sanitized_lib):
    r = _drive(sanitized_lib, "clean")
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-3000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-3000:]
    assert int(out.split("checked")[1].split()[0]) > 24000


def test_the_harness_reports_an_overflow(sanitized_lib):
    # gs_features given one row less than the candidates it must write
    r = _drive(sanitized_lib, "overflow")
    assert r.returncode != 0
    assert "AddressSanitizer" in r.stdout + r.stderr
