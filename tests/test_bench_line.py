"""The bench line on CPU: bench_line() assembles the contract's JSON line
from one workload's measurements, here fake ones with round numbers, so
that every key and every derived figure is checked without a GPU."""
import argparse
import json
import math

import pytest

import bench


def _fake(w, launches):
    return dict(S=100, depth=1, graph_ms=[3.0, 3.2, 3.1, 2.9], per_step_ms=[6.0, 6.2, 6.1, 5.9], kern_ms=0.0025,
                e2e=(0.004, 9_437_184, 8_388_608), paper_conv_ms=30.0, build_s=0.01, launches=launches)


@pytest.mark.parametrize("workload", sorted(bench.WORKLOADS))
def test_bench_line_keys_and_arithmetic(workload):
    w = bench.WORKLOADS[workload]
    args = argparse.Namespace(steps=4, warmup=3, workload=workload)
    launches = 2 * w["iters"] if w["kind"] == "fdtd" else w["iters"]
    m = _fake(w, launches)
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    line = bench.bench_line(args, w, m, clk, 1)
    json.dumps(line)  # serialisable
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    for k in ("h2d_bytes_per_step", "d2h_bytes_per_step", "value", "unit"):
        assert k in line["e2e"], k
    assert line["config"]["workload"] == workload and "seed" in line["config"]
    units = bench.cells_of(w) * w["iters"]
    total_ms = sum(m["graph_ms"])
    assert math.isclose(line["value"], units * 4 / (total_ms * 1e-3), rel_tol=1e-12)
    assert math.isclose(line["ms_per_step"], total_ms / 4, rel_tol=1e-12)
    launch_ms = total_ms / 4 / launches
    achieved = bench.algo_bytes_per_launch(w, 1) / (launch_ms * 1e-3) / 1e9
    rf = line["roofline"]
    assert math.isclose(rf["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(rf["frac"], achieved / rf["peak"], rel_tol=1e-12)
    assert math.isclose(rf["frac_of_nominal"], achieved / bench.NOMINAL_HBM_GBS, rel_tol=1e-12)
    assert rf["traffic"] is None or isinstance(rf["traffic"], int)
    # the bound follows the working set against the L2 size (fake: 126 MiB)
    assert rf["bound"] == ("hbm" if bench.working_set_bytes(w) > 63 * 2 ** 20 else "l2/latency")
    assert math.isclose(rf["per_node_us"], launch_ms * 1e3, rel_tol=1e-12)
    assert math.isclose(line["e2e"]["value"], units / 0.004, rel_tol=1e-12)
    assert line["gpu_launches"] == launches * 4
    assert math.isclose(line["ms_per_step_std"], 0.1118033988749895, rel_tol=1e-9)  # pstdev of 3.0, 3.2, 3.1, 2.9
    assert math.isclose(line["per_step_launch"]["ms_per_step_std"], 0.1118033988749895, rel_tol=1e-9)
    assert math.isclose(line["per_step_launch"]["graph_speedup"], line["value"] / (units / 6.05e-3), rel_tol=1e-12)


def test_bounds_of_the_named_workloads():
    # L2 126 MiB: the 3D 512x512x8 field (17 MiB) and FDTD 128^3 (53 MB) stay
    # in L2; 2D 4096^2 (192 MiB), 256^3 and the 64-grid batch (141 MB) do not
    half = 63 * 2 ** 20
    ws = {k: bench.working_set_bytes(w) for k, w in bench.WORKLOADS.items()}
    assert ws["heat3d-512x512x8"] < half and ws["fdtd-128"] < half and ws["heat2d-512"] < half
    for k in ("heat2d-4096", "heat3d-256", "fdtd-256", "fdtd-media-256", "multi-64"):
        assert ws[k] > half, k


def test_hbm_roofline_of_arithmetic():
    w = bench.WORKLOADS["heat2d-4096"]
    mm = dict(S=100, depth=1, graph_ms=[5.2, 5.4], launches=200)
    r = bench.hbm_roofline_of("heat2d-4096", w, mm)
    bl = 4096 * 4096 * 12
    assert r["bytes_per_launch"] == bl and r["bound"] == "hbm"
    assert math.isclose(r["achieved"], bl / (5.3e-3 / 200) / 1e9, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-12)
    if r["traffic"] is not None and "cold_cache_us" in r:
        assert math.isclose(r["cold_cache_frac"], bl / (r["cold_cache_us"] * 1e-6) / 1e9 / r["peak"], rel_tol=1e-12)


def test_column_geometry_of_the_default_workload():
    # 3D 512x512x8, COLUMN rows 4: 4 x 128 blocks of 32 x 4 threads
    assert bench.column_geometry(bench.WORKLOADS["heat3d-512x512x8"], dict(kernel=4, rows=4), 1) == (512, 128)
    # at depth 2 (block_x 64): 19 x 64 blocks of 32 x 2 threads (28 cells, 4 rows a warp)
    assert bench.column_geometry(bench.WORKLOADS["heat3d-512x512x8"], dict(kernel=4, block_x=64), 2) == (1216, 64)
    assert bench.column_geometry(bench.WORKLOADS["fdtd-128"], dict(kernel=4), 1) is None


def test_profiles_hold_the_default_workloads_traffic_line():
    # roofline.traffic comes from a committed ncu summary's line
    # "bench-traffic: workload=W kernel=K sha256=H bytes=B"; the bench takes it
    # only while H is the hash of the current kernel sources
    import glob
    import os
    import re

    found = []
    for path in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")):
        with open(path) as f:
            found += re.findall(r"^bench-traffic: workload=(\S+) kernel=\S+ sha256=(\w{16}) bytes=(\d+)(?: us=\S+)?$", f.read(),
                                flags=re.M)
    mine = [f for f in found if f[0] == bench.DEFAULT]
    assert mine, "no bench-traffic line for the default workload under profiles/"
    rec = bench.recorded_traffic(bench.DEFAULT)
    assert rec is None or rec in [int(b) for _, _, b in mine]
    if rec is not None:  # no gross re-reads (an L2-resident workload reads less than its algorithmic bytes)
        assert 0 < rec <= 1.5 * bench.algo_bytes_per_launch(bench.WORKLOADS[bench.DEFAULT], 1)


def test_oracle_single_thread_figure_restores_the_thread_count():
    import oracle

    every = oracle.num_threads()
    r = bench.oracle_single_thread(bench.WORKLOADS["heat2d-512"], budget_s=0.05)
    assert r["cores"] == 1 and r["value"] > 0 and "first" in r["sample"]
    assert oracle.num_threads() == every
