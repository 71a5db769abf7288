"""The bounds-checked build (GS_CHECKED) on the small parity shapes: every
global field access of every thermal and FDTD kernel variant, and of the
instance-batch kernel, lies inside a registered buffer (no access refused),
and the checked build's results equal the ordinary build's bit for bit.  A
planted case leaves the power map's buffer out of the table and must see
its loads refused.  This ties the CPU re-traces of the kernels' index
arithmetic (test_kernel_index_bounds.py) to the kernels themselves; the
checked library runs in a process of its own."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


def test_checked_build_refuses_nothing_and_changes_nothing(tmp_path):
    import torch

    import __graft_entry__
    import paper_2501_09398_gb300 as g

    __graft_entry__._builder().build(checked=True)
    npz, js = str(tmp_path / "out.npz"), str(tmp_path / "refused.json")
    env = dict(os.environ, GS_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py"), npz, js], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    with open(js) as f:
        refused = json.load(f)
    planted = refused.pop("planted: P not registered")
    bad = {k: v for k, v in refused.items() if v[0] != 0}
    assert not bad, bad
    assert planted[0] > 0 and planted[2] <= planted[1] < planted[3], planted
    got = np.load(npz)
    sys.path.insert(0, HERE)
    from checked_cases import cases

    torch.cuda.set_stream(torch.cuda.Stream())
    assert not g.gs_debug_checked_build()
    n = 0
    for name, fn in cases():
        outs, _, _ = fn(g)
        for k, o in enumerate(outs):
            assert np.array_equal(got[f"{name}#{k}"], o), (name, k)
            n += 1
    assert n >= 100
