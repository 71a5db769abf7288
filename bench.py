#!/usr/bin/env python
"""Benchmark: graph-batched stencil time stepping vs per-step launch on GB300.

Default workload: 3D thermal 7-point stencil, 512x512x8 FP32, 1000
iterations per step, seeded synthetic T ~ U[320,340], P ~ U[0,1e-3] on
layer 0.  One bench "step" is one whole 1000-iteration run of the workload
through the library's graph-batched path (gs_step with batch size S).
L2 is flushed (256 MiB write) between timed steps, outside the timed events.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (the only comparison program there is:
the paper ships no code).

Other workloads (``--workload``): heat2d-512 (2D 512^2, 1000 iterations),
heat2d-4096 (2D 4096^2, 200 iterations), heat3d-256 (a deep stack, 256^3,
200 iterations), fdtd-128 (Yee 128^3, 5000 iterations), fdtd-256 and
fdtd-media-256 (256^3 cavities, vacuum and lossy objects, 500 iterations),
multi-64 (64 uneven 2D grids, 2000 iterations).  The default run adds a
line's "extra" measurements of several of these (and of temporal depths),
and the batch-size sweep S = 1 ... 1000 of the 2D 512^2 and 3D 512x512x8
workloads at temporal depths 1, 2 and 4.
Multi-GPU (torchrun): independent replicas, one per rank, no collective on
the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gs_inputs  # noqa: E402

# Default launch plans per workload (the fastest measured on GB300; the
# autotuner can re-derive them).  kernel: 1 = MARCH, 2 = WAVE, 4 = COLUMN.
# The per-step baseline always uses plain launches (use_pdl forced off).
WORKLOADS = {
    # temporal depth 2: the register COLUMN kernel advances two steps per
    # launch, with programmatic-dependent-launch edges between the graph's
    # nodes (measured 7.29e11 cell-updates/s; 6.95e11 without the edges,
    # 6.78e11 at depth 1, where the edges cost 5 %)
    "heat3d-512x512x8": dict(kind="heat3d", nx=512, ny=512, nz=8, iters=1000, S=100, depth=2,
                             plan=dict(kernel=4, block_x=64, use_pdl=1)),
    # a deep stack (nz > 8): the column kernel in 8-plane chunks
    "heat3d-256": dict(kind="heat3d", nx=256, ny=256, nz=256, iters=200, S=100, depth=1,
                       plan=dict(kernel=4, rows=4)),
    "heat2d-512": dict(kind="heat2d", nx=512, ny=512, nz=1, iters=1000, S=100, depth=1,
                       plan=dict(kernel=4, rows=4)),
    "heat2d-4096": dict(kind="heat2d", nx=4096, ny=4096, nz=1, iters=200, S=100, depth=1,
                        plan=dict(kernel=4, rows=8)),
    "fdtd-128": dict(kind="fdtd", N=128, iters=5000, S=100, depth=1, plan=dict(kernel=4, rows=2)),
    # larger cavities (HBM-bound), in vacuum and filled with lossy objects
    "fdtd-256": dict(kind="fdtd", N=256, iters=500, S=100, depth=1, plan=dict(kernel=4, rows=2)),
    "fdtd-media-256": dict(kind="fdtd", N=256, iters=500, S=100, depth=1, plan=dict(kernel=4, rows=2),
                           media=dict(n_mat=8, n_boxes=24, seed=0)),
    # the fused plan comes from gs_multi_autotune over the library's candidates
    # at S = 100 (tune=True); plan/depth are the fallback when a flag overrides
    "multi-64": dict(kind="multi", n=64, lo=64, hi=1024, iters=2000, S=100, depth=2, plan=dict(kernel=4, rows=2),
                     tune=True),
}
DEFAULT = "heat3d-512x512x8"
METRIC = "cell-updates/s (graph-batched)"
FLUSH_BYTES = 256 << 20
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, vendor figure (context beside the measured copy peak)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def multi_sides(w):
    return gs_inputs.instance_sides(w["n"], w["lo"], w["hi"], seed=0)


def kernel_sha():
    """First 16 hex digits of sha256 over the thermal kernel sources with
    their comments and blank lines removed (so an edit of a comment keeps a
    capture valid)."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in ("heat.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2501_09398_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(src.encode())
    return h.hexdigest()[:16]


def recorded_capture(workload):
    """(DRAM bytes, cold-cache microseconds or None) per launch from the
    committed ncu summaries, if they were taken on the current kernel
    sources (else (None, None))."""
    import glob
    import re

    sha = kernel_sha()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = re.match(r"bench-traffic: workload=(\S+) kernel=\S+ sha256=(\w+) bytes=(\d+)(?: us=(\S+))?", line)
                if m and m.group(1) == workload and m.group(2) == sha:
                    return int(m.group(3)), (float(m.group(4)) if m.group(4) else None)
    return None, None


def recorded_traffic(workload):
    """DRAM bytes per launch from the committed ncu summaries, if they were
    taken on the current kernel sources (else None)."""
    return recorded_capture(workload)[0]


def cells_of(w):
    if w["kind"] == "multi":
        return sum(s * s for s in multi_sides(w))
    return w["N"] ** 3 if w["kind"] == "fdtd" else w["nx"] * w["ny"] * w["nz"]


def algo_bytes_per_launch(w, depth, elem=4, fused=False):
    """Algorithmic DRAM bytes of one kernel launch.

    Thermal depth-t launch: read T once, write T once, read the P plane once
    (2D: P is the full plane), for t cell-updates per cell.  FDTD half-step
    (H or E kernel): read 6 components, write 3, per cell, plus the 1-byte
    material id in media; fused FDTD step (one launch per step): read 6
    components and write 6 (and the id once in media)."""
    if w["kind"] == "fdtd":
        if fused:
            return cells_of(w) * (12 * elem + (1 if w.get("media") else 0))
        return cells_of(w) * (9 * elem + (1 if w.get("media") else 0))
    if w["kind"] == "multi":
        return cells_of(w) * 3 * elem
    plane = w["nx"] * w["ny"]
    return cells_of(w) * 2 * elem + plane * elem


def working_set_bytes(w, elem=4):
    """Bytes one step touches: both thermal buffers and the power map; the
    six FDTD components (and the material map); every instance's fields."""
    if w["kind"] == "fdtd":
        m = (w["N"] + 1) ** 3
        return m * (6 * elem + (1 if w.get("media") else 0))
    if w["kind"] == "multi":
        return cells_of(w) * 3 * elem
    return cells_of(w) * 2 * elem + w["nx"] * w["ny"] * elem


def column_geometry(w, plan, depth):
    """(blocks, threads per block) of the thermal COLUMN kernel's launch for
    this workload and plan (the launch shapes of heat_desc), else None."""
    if w["kind"] not in ("heat2d", "heat3d") or plan.get("kernel", 4) != 4:
        return None
    cdiv = lambda a, b: -(-a // b)  # noqa: E731
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    if depth > 1:
        bw = max(1, min(plan.get("block_x", 64) // 32, 8))
        if w["kind"] == "heat3d":  # one cell a lane, 32 - 2t stored; R rows a warp
            if nz > 8:
                return None
            R = 4 if (depth == 2 and plan.get("rows", 0) != 2) else 2
            return cdiv(nx, 32 - 2 * depth) * cdiv(ny, R * bw), 32 * bw
        return cdiv(nx, 30 * 4) * cdiv(ny, 4 * bw), 32 * bw
    by = max(1, min(plan.get("rows", 4), 8))
    cw = 4  # cells per thread in f32 (2D: one 16-byte vector; 3D: four cells)
    chunks = cdiv(nz, 8) if nz > 8 else 1
    return cdiv(nx, 32 * cw) * cdiv(ny, by) * chunks, 32 * by


def graph_node_floor_us(blocks, threads, flush, nodes=100, launches=10):
    """Per-node time of a graph of `nodes` skeleton-kernel nodes launched on
    `blocks` blocks of `threads` threads, each thread scaling one 16-byte
    vector in place (an L2-resident field): what one graph node of that
    launch shape costs when its kernel does almost nothing."""
    import torch

    import paper_2501_09398_gb300 as g

    n = blocks * threads * 4
    st = torch.cuda.current_stream()
    ctx = g.gs_create(g.GS_SKELETON, n, 1, 1, g.GS_F32, g.GS_BC_CLAMP, st.cuda_stream)
    x = torch.ones(n, dtype=torch.float32, device="cuda")
    try:
        g.gs_bind_field(ctx, g.GS_FIELD_X, x.data_ptr(), n)
        g.gs_set_plan(ctx, block_x=threads)
        g.gs_step(ctx, nodes, nodes)  # builds the graph
        times = []
        for _ in range(5):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            g.gs_step(ctx, nodes * launches, nodes)
            b.record(st)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    finally:
        g.gs_destroy(ctx)
    return statistics.median(times) * 1e3 / (nodes * launches)


def l2_bytes():
    import torch

    v = getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "L2_cache_size", 0)
    return int(v) if v else 126 << 20


# ------------------------------------------------------------ clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        if os.environ.get("CUDA_INJECTION64_PATH"):
            # under a profiler's injection (ncu): numbers from such a run are
            # not bench values, and the sampler would poll NVML during capture
            self.proc = None
            self.skipped = True
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            why = "not sampled under a profiler" if getattr(self, "skipped", False) else "nvidia-smi unavailable"
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [why]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _smi_id():
    import torch

    try:
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis if vis.isdigit() else "0"


# ------------------------------------------------------- oracle timing --
def oracle_sample(w, budget_s=10.0):
    """Time the FP64 oracle on a bounded sample of the workload.

    Returns (cell-updates/s, sample description, threads, oracle result of
    the full workload if it was run in full, else None)."""
    import oracle

    oracle.build()
    threads = oracle.num_threads()
    if w["kind"] == "fdtd":
        N = w["N"]
        f = oracle.fdtd_zero_fields(N)
        media = gs_inputs.fdtd_media(N, **w["media"]) if w.get("media") else None
        n = 0
        t0 = time.perf_counter()
        chunk = 20
        while n < w["iters"] and time.perf_counter() - t0 < budget_s:
            oracle.fdtd_run(f, N, chunk, n0=n, src=(N // 2, N // 2, N // 2), media=media)
            n += chunk
        dt = time.perf_counter() - t0
        full = f if n >= w["iters"] else None
        what = "FDTD in media" if media else "FDTD"
        return cells_of(w) * n / dt, f"{what} {N}^3, first {n} of {w['iters']} steps", threads, full
    if w["kind"] == "multi":
        sides = multi_sides(w)
        fields = gs_inputs.instance_fields(sides)
        n = 0
        done = 0
        t0 = time.perf_counter()
        for (T, P) in fields:  # whole instances, smallest work first order as generated
            if time.perf_counter() - t0 > budget_s:
                break
            oracle.heat_run(T, P, w["iters"], oracle.HEAT_COEFFS_2D)
            n += T.size * w["iters"]
            done += 1
        dt = time.perf_counter() - t0
        return n / dt, f"{done} of {len(sides)} instances, {w['iters']} iterations each", threads, None
    T0, P = gs_inputs.heat_fields(w["nx"], w["ny"], w["nz"], seed=0)
    coeffs = oracle.HEAT_COEFFS_2D if w["nz"] == 1 else oracle.HEAT_COEFFS_3D
    T = T0
    n = 0
    chunk = 50
    t0 = time.perf_counter()
    while n < w["iters"] and time.perf_counter() - t0 < budget_s:
        T = oracle.heat_run(T, P, chunk, coeffs)
        n += chunk
    dt = time.perf_counter() - t0
    full = T if n >= w["iters"] else None
    shape = "x".join(str(v) for v in (w["nx"], w["ny"], w["nz"]))
    return cells_of(w) * n / dt, f"thermal {shape}, first {n} of {w['iters']} iterations", threads, full


def oracle_single_thread(w, budget_s=5.0):
    """The oracle's throughput on one host thread (a shorter bounded sample
    of the same workload), beside its all-cores figure."""
    import oracle

    every = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        v, sample, threads, _ = oracle_sample(w, budget_s=budget_s)
    finally:
        oracle.set_num_threads(every)
    return {"value": v, "unit": "cell-updates/s", "cores": threads, "sample": sample}


def config_of(name, w, S, depth, world):
    """The bench line's config (same keys on both arms), with the seeds of
    its synthetic inputs."""
    if w["kind"] == "multi":
        seed = "sides: seed 0; instance k fields: seed 1000 + k"
    elif w["kind"] == "fdtd":
        seed = "fields start at 0 (source-driven); media: seed %d" % w["media"]["seed"] if w.get("media") else \
            "none: fields start at 0 (source-driven)"
    else:
        seed = 0
    return {"workload": name, "iterations_per_step": w["iters"], "batch_size_S": S, "temporal_depth": depth,
            "parallelism": f"replicas x{world}" if world > 1 else "single",
            "l2": "flushed between steps (256 MiB write)", "seed": seed}


def aggregate(step_ms, units_per_step, group=None):
    """Whole-job throughput of independent replicas: each rank timed its own
    steps (step_ms, device milliseconds); the job time is the maximum over
    ranks of their summed step times and the work is every rank's units.
    Returns (value in units/s, job milliseconds, world size)."""
    import torch

    world = 1
    total = float(sum(step_ms))
    if group is not None or (torch.distributed.is_available() and torch.distributed.is_initialized()):
        import torch.distributed as dist

        world = dist.get_world_size(group)
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.tensor([total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        total = float(t.item())
    return world * units_per_step * len(step_ms) / (total * 1e-3), total, world


def run_reference(args, w, name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    sample = threads = None
    for i in range(args.warmup + args.steps):
        v, sample, threads, _ = oracle_sample(w, budget_s=max(1.0, 60.0 / (args.warmup + args.steps)))
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cells_of(w) * w["iters"] / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(name, w, w["S"], w["depth"], args.gpus),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm --
class Runner:
    """One workload bound to a context on the current torch stream."""

    def __init__(self, w, S, depth, plan_extra):
        import torch

        import paper_2501_09398_gb300 as g

        self.g, self.w, self.S, self.depth = g, w, S, depth
        self.stream = torch.cuda.current_stream()
        h = self.stream.cuda_stream
        if w["kind"] == "fdtd":
            N = w["N"]
            self.ctx = g.gs_create(g.GS_FDTD3D, N, N, N, g.GS_F32, g.GS_BC_PEC, h)
            self.fields = g.FdtdFields(self.ctx, N, media=bool(w.get("media")))
            g.gs_set_fdtd_params(self.ctx, courant=0.5, src_on=1, src=(N // 2, N // 2, N // 2))
            if w.get("media"):
                mat, table = gs_inputs.fdtd_media(N, **w["media"])
                g.gs_set_fdtd_media(self.ctx, table)
                g.gs_upload_u8(self.ctx, g.GS_FIELD_MAT, mat)
            self.host_in = []
            self.out_shape = (N + 1,) * 3
        else:
            kind = g.GS_HEAT2D if w["kind"] == "heat2d" else g.GS_HEAT3D
            self.ctx = g.gs_create(kind, w["nx"], w["ny"], w["nz"], g.GS_F32, g.GS_BC_CLAMP, h)
            self.fields = g.HeatFields(self.ctx, w["nx"], w["ny"], w["nz"])
            T0, P = gs_inputs.heat_fields(w["nx"], w["ny"], w["nz"], seed=0)
            self.T0, self.P = T0, P
            self.out_shape = T0.shape
        plan = dict(temporal_depth=depth, **plan_extra)
        g.gs_set_plan(self.ctx, **plan)
        self.fused = plan.get("kernel") == g.GS_KERNEL_FUSED
        self.reset()

    def reset(self):
        g = self.g
        if self.w["kind"] == "fdtd":
            z = np.zeros(self.out_shape, dtype=np.float32)
            for fid in g.FDTD_FIELDS:
                g.gs_upload(self.ctx, fid, z)
            g.gs_set_time(self.ctx, 0)
        else:
            g.gs_upload(self.ctx, g.GS_FIELD_T, self.T0)
            g.gs_upload(self.ctx, g.GS_FIELD_P, self.P)

    def step(self, S):
        self.g.gs_step(self.ctx, self.w["iters"], S)

    def read(self):
        g = self.g
        if self.w["kind"] == "fdtd":
            return [g.gs_read_field(self.ctx, fid, np.empty(self.out_shape, dtype=np.float32)) for fid in g.FDTD_FIELDS]
        return g.gs_read_field(self.ctx, g.GS_FIELD_T, np.empty(self.out_shape, dtype=np.float32))

    def launches_per_step(self, S):
        it = self.w["iters"]
        if self.w["kind"] == "fdtd":
            return it + (it & 1) if self.fused else 2 * it
        t = self.depth
        return it // t + it % t

    def close(self):
        self.g.gs_destroy(self.ctx)


class MultiRunner:
    """The uneven-instance batch: fused persistent kernel in captured graphs
    (S > 0) against 64 separate per-step launch loops (S = 0)."""

    def __init__(self, w, S, depth, plan_extra, tune=False):
        import torch

        import paper_2501_09398_gb300 as g

        self.g, self.w, self.S, self.depth = g, w, S, 1
        self.stream = torch.cuda.current_stream()
        self.sides = multi_sides(w)
        self.m = g.gs_multi_create(self.sides, self.sides, g.GS_F32, g.GS_BC_CLAMP, self.stream.cuda_stream)
        self.ctx = None
        self.fields = g.MultiFields(self.m, self.sides, self.sides)
        self.inputs = gs_inputs.instance_fields(self.sides)
        self.reset()
        self.tuned = None
        if tune:
            # the fused plan the batch's tuner picks for a whole run at this S
            cands = [(p, s) for p, s in g.gs_multi_candidates(self.m) if s == S]
            res, best = g.gs_multi_autotune(self.m, w["iters"], cands, reps=2)
            self.tuned = dict(res[best]["plan"])
            self.tuned["candidates"] = len(cands)
            g.gs_multi_set_plan(self.m, **{k: v for k, v in res[best]["plan"].items()})
            self.depth = res[best]["plan"]["temporal_depth"]
            return
        mp = {k: v for k, v in plan_extra.items() if k in ("block_x", "rows", "use_pdl", "kernel", "traverse")}
        if depth > 1:
            mp["temporal_depth"] = depth
            self.depth = depth
        if mp:
            g.gs_multi_set_plan(self.m, **mp)

    def reset(self):
        g = self.g
        for i, (T, P) in enumerate(self.inputs):
            g.gs_multi_upload(self.m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(self.m, i, g.GS_FIELD_P, P)

    def step(self, S):
        g = self.g
        if S == 0:
            g.gs_multi_step(self.m, self.w["iters"], 0, g.GS_MULTI_SEPARATE)
        else:
            g.gs_multi_step(self.m, self.w["iters"], S, g.GS_MULTI_FUSED)

    def one_launch(self):
        self.g.gs_multi_step(self.m, self.depth, 0, self.g.GS_MULTI_FUSED)

    def read(self):
        g = self.g
        return [g.gs_multi_read_field(self.m, i, g.GS_FIELD_T, np.empty_like(T)) for i, (T, _) in
                enumerate(self.inputs)]

    def launches_per_step(self, S):
        it, t = self.w["iters"], self.depth
        return (it // t + it % t) if S > 0 else it * len(self.sides)

    def graph_build(self, S):
        self.step(S)  # first use captures the graphs

    def close(self):
        self.g.gs_multi_destroy(self.m)


def timed_steps(run, S, K, W, flush):
    """Device time of K steps (CUDA events on the launching stream), L2
    flushed between steps outside the events.  Returns per-step ms list."""
    import torch

    st = run.stream
    for _ in range(W):
        flush.zero_()
        run.step(S)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in evs:
        flush.zero_()
        a.record(st)
        run.step(S)
        b.record(st)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def kernel_avg_ms(run, flush, reps=6, per=16):
    """Average duration of one launch of the dominant kernel: events around
    single launches queued behind an L2-flush write so the GPU runs them back
    to back (the host enqueues ahead while the flush runs)."""
    import torch

    g = run.g
    st = run.stream
    fused = bool(getattr(run, "fused", False))
    n_iter = (2 if fused else 1) if run.w["kind"] == "fdtd" else run.depth
    times = []
    for _ in range(reps):
        flush.zero_()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(per)]
        for a, b in evs:
            a.record(st)
            if run.w["kind"] == "multi":
                run.one_launch()
            else:
                g.gs_step(run.ctx, n_iter, 0)
            b.record(st)
        torch.cuda.synchronize()
        times += [a.elapsed_time(b) for a, b in evs]
    # FDTD: one gs_step(1) is an H launch and an E launch, one fused
    # gs_step(2) two fused launches; report per launch
    div = 2 if run.w["kind"] == "fdtd" else 1
    return statistics.median(times) / div


def e2e_steps(run, S, K):
    """Wall time per step through the public API with host buffers: upload
    inputs from pinned host memory, step, read the result back."""
    import torch

    g = run.g
    if run.w["kind"] == "multi":
        pins = [(torch.from_numpy(T).pin_memory().numpy(), torch.from_numpy(P).pin_memory().numpy())
                for T, P in run.inputs]
        outs = [torch.empty(T.shape, dtype=torch.float32).pin_memory().numpy() for T, _ in run.inputs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            for i, (T, P) in enumerate(pins):
                g.gs_multi_upload(run.m, i, g.GS_FIELD_T, T)
                g.gs_multi_upload(run.m, i, g.GS_FIELD_P, P)
            run.step(S)
            for i, o in enumerate(outs):
                g.gs_multi_read_field(run.m, i, g.GS_FIELD_T, o)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / K
        return dt, sum(T.nbytes + P.nbytes for T, P in pins), sum(o.nbytes for o in outs)
    if run.w["kind"] == "fdtd":
        hz = torch.zeros(run.out_shape, dtype=torch.float32).pin_memory().numpy()
        h_in = [hz] * 6
        fids = list(g.FDTD_FIELDS)
    else:
        h_in = [torch.from_numpy(run.T0).pin_memory().numpy(), torch.from_numpy(run.P).pin_memory().numpy()]
        fids = [g.GS_FIELD_T, g.GS_FIELD_P]
    h_out = torch.empty(run.out_shape, dtype=torch.float32).pin_memory().numpy()
    out_fid = g.GS_FIELD_EZ if run.w["kind"] == "fdtd" else g.GS_FIELD_T
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        for fid, h in zip(fids, h_in):
            g.gs_upload(run.ctx, fid, h)
        if run.w["kind"] == "fdtd":
            g.gs_set_time(run.ctx, 0)
        run.step(S)
        g.gs_read_field(run.ctx, out_fid, h_out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / K
    h2d = sum(h.nbytes for h in h_in)
    return dt, h2d, h_out.nbytes


def measure_workload(name, w, args, flush, with_e2e=True):
    import torch

    g_plan = dict(w.get("plan", {}))
    if args.block_x:
        g_plan["block_x"] = args.block_x
    if args.rows:
        g_plan["rows"] = args.rows
    if args.tile_x:
        g_plan["tile_x"] = args.tile_x
    if args.tile_y:
        g_plan["tile_y"] = args.tile_y
    if args.pdl:
        g_plan["use_pdl"] = 1
    if getattr(args, "kernel", 0):
        g_plan["kernel"] = args.kernel
    if getattr(args, "loop", False):
        g_plan["graph_loop"] = 1
    if getattr(args, "traverse", 0):
        g_plan["traverse"] = args.traverse
    S = args.batch or w["S"]
    depth = args.depth or w["depth"]
    if w["kind"] == "multi":
        overridden = args.depth or args.block_x or args.rows or getattr(args, "kernel", 0) or args.pdl
        run = MultiRunner(w, S, depth, g_plan, tune=bool(w.get("tune")) and not overridden)
        depth = run.depth
    else:
        run = Runner(w, S, depth, g_plan)
    try:
        g = run.g
        # paper convention (Sec. III-C): graph creation + execution of one run
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if run.ctx is not None:
            g.gs_graph_destroy(run.ctx)
            g.gs_graph_build(run.ctx, S)
            run.step(S)
        else:
            run.graph_build(S)
        torch.cuda.synchronize()
        paper_conv_ms = (time.perf_counter() - t0) * 1e3
        build_s = g.gs_get_stats(run.ctx)["last_build_seconds"] if run.ctx is not None else None
        # steady state (graphs cached)
        graph_ms = timed_steps(run, S, args.steps, args.warmup, flush)
        # the per-step baseline is the paper's Listing 1: plain launches
        if g_plan.get("use_pdl") and run.ctx is not None:
            g.gs_set_plan(run.ctx, temporal_depth=depth, **{k: v for k, v in g_plan.items() if k != "use_pdl"})
        per_step_ms = timed_steps(run, 0, args.steps, args.warmup, flush)
        if g_plan.get("use_pdl") and run.ctx is not None:
            g.gs_set_plan(run.ctx, temporal_depth=depth, **g_plan)
            g.gs_graph_build(run.ctx, S)
        kern_ms = kernel_avg_ms(run, flush)
        e2e = e2e_steps(run, S, max(3, min(args.steps, 20))) if with_e2e else None
        l2 = l2_bytes()
        floor = None
        geo = column_geometry(w, g_plan, depth)
        if with_e2e and geo is not None and working_set_bytes(w) <= 0.5 * l2:
            floor = graph_node_floor_us(geo[0], geo[1], flush)
        # result after one clean run, for the error check
        run.reset()
        run.step(S)
        result = run.read()
    finally:
        run.close()
    return dict(S=S, depth=depth, graph_ms=graph_ms, per_step_ms=per_step_ms, kern_ms=kern_ms, e2e=e2e,
                fused=bool(getattr(run, "fused", False)),
                paper_conv_ms=paper_conv_ms, build_s=build_s, result=result,
                launches=run.launches_per_step(S), l2_bytes=l2, node_floor_us=floor,
                tuned_plan=getattr(run, "tuned", None), plan=g_plan)


SWEEP_S = (1, 10, 50, 100, 500, 1000)
# (temporal depth, launch plan) per swept workload: depth 1 is the bench's
# COLUMN plan; depths 2 and 4 run the register COLUMN kernel (2D, and stacks
# of up to eight planes); the 3D sweep also keeps the shared-memory WAVE
# kernel at depth 2 for comparison
SWEEP_PLANS = {
    "heat2d-512": ((1, dict(kernel=4, block_x=64, rows=4)), (2, dict(kernel=4, block_x=64, rows=4)),
                   (4, dict(kernel=4, block_x=64, rows=4))),
    "heat3d-512x512x8": ((1, dict(kernel=4, block_x=64, rows=4)), (2, dict(kernel=4, block_x=64)),
                         (4, dict(kernel=4, block_x=64)), (2, dict(kernel=2, block_x=64, rows=4))),
}


def batch_sweep(w, plans, flush, steps=10, warmup=3):
    """Cell-updates/s of one workload's whole run at every batch size of the
    sweep (each graph built during the warm-up, outside the timing) beside
    per-step launch of the same kernels, for each (temporal depth, plan)."""
    units = cells_of(w) * w["iters"]
    out = {}
    for depth, plan in plans:
        run = Runner(w, 0, depth, plan)
        try:
            row = {"plan": dict(plan),
                   "per_step": units / (statistics.mean(timed_steps(run, 0, steps, warmup, flush)) * 1e-3)}
            for S in SWEEP_S:
                row[f"S={S}"] = units / (statistics.mean(timed_steps(run, S, steps, warmup, flush)) * 1e-3)
        finally:
            run.close()
        best = max(SWEEP_S, key=lambda s: row[f"S={s}"])
        row["best_S"] = best
        row["best_vs_per_step"] = row[f"S={best}"] / row["per_step"]
        key = f"depth{depth}" if f"depth{depth}" not in out else f"depth{depth}/kernel{plan.get('kernel', 0)}"
        out[key] = row
    return out


def multi_streams_per_step(w, flush, reps=5, warmup=2):
    """The instance batch's per-step baseline with one stream per instance:
    a context per grid (default plan) on its own stream, each stepped by
    plain per-step launches, issued instance after instance; the GPU may
    overlap the streams.  Device time from an event on the launching stream
    (every instance stream waits on it) to one recorded after the launching
    stream has waited on every instance stream."""
    import torch

    import paper_2501_09398_gb300 as g

    sides = multi_sides(w)
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in sides]
    ctxs, keep = [], []
    try:
        for s, st, (T, P) in zip(sides, streams, gs_inputs.instance_fields(sides)):
            c = g.gs_create(g.GS_HEAT2D, s, s, 1, g.GS_F32, g.GS_BC_CLAMP, st.cuda_stream)
            ctxs.append(c)
            keep.append(g.HeatFields(c, s, s, 1))
            g.gs_upload(c, g.GS_FIELD_T, T)
            g.gs_upload(c, g.GS_FIELD_P, P)
        torch.cuda.synchronize()
        times = []
        for r in range(warmup + reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            for st in streams:
                st.wait_stream(main)
            for c in ctxs:
                g.gs_step(c, w["iters"], 0)
            for st in streams:
                main.wait_stream(st)
            b.record(main)
            torch.cuda.synchronize()
            if r >= warmup:
                times.append(a.elapsed_time(b))
    finally:
        for c in ctxs:
            g.gs_destroy(c)
    ms = statistics.mean(times)
    return {"value": cells_of(w) * w["iters"] / (ms * 1e-3), "ms": ms, "ms_std": statistics.pstdev(times),
            "streams": len(streams), "launches": len(sides) * w["iters"], "plan": "each context's default (COLUMN)"}


def fdtd_precision(N=128, iters=5000, S=100):
    """Relative L2 error (six components concatenated) of the driven 128^3
    cavity after 5000 steps against the FP64 oracle, for each storage type,
    with the bar the arithmetic gives for bf16/f16 storage (two roundings per
    step, unbiased: 2 sqrt(n) u)."""
    import math

    import torch

    import oracle
    import paper_2501_09398_gb300 as g

    src = (N // 2, N // 2, N // 2)
    ref = oracle.fdtd_run(oracle.fdtd_zero_fields(N), N, iters, src=src)
    refv = np.concatenate([ref[c].ravel() for c in oracle.FDTD_COMPONENTS])
    stream = torch.cuda.current_stream().cuda_stream
    out = {"workload": f"FDTD {N}^3 driven cavity, {iters} steps, S = {S}"}
    for name, dt, u in (("f32", g.GS_F32, 2.0 ** -24), ("bf16", g.GS_BF16, 2.0 ** -8), ("f16", g.GS_F16, 2.0 ** -11)):
        ctx = g.gs_create(g.GS_FDTD3D, N, N, N, dt, g.GS_BC_PEC, stream)
        fields = g.FdtdFields(ctx, N, dt)
        try:
            g.gs_set_fdtd_params(ctx, courant=0.5, src_on=1, src=src)
            z = np.zeros((N + 1,) * 3, dtype=np.float32)
            for fid in g.FDTD_FIELDS:
                g.gs_upload(ctx, fid, z)
            g.gs_step(ctx, iters, S)
            got = np.concatenate([g.gs_read_field(ctx, fid, np.empty((N + 1,) * 3, dtype=np.float32))
                                  .astype(np.float64).ravel() for fid in g.FDTD_FIELDS])
        finally:
            g.gs_destroy(ctx)
            del fields
        err = float(np.linalg.norm(got - refv) / np.linalg.norm(refv))
        out[name] = {"rel_l2": err, "bar": 1e-4 if name == "f32" else 2.0 * math.sqrt(iters) * u}
    return out


def error_vs_oracle(w, result, full_ref):
    if full_ref is None:
        return None
    if w["kind"] == "fdtd":
        import oracle

        ref = np.concatenate([full_ref[c].ravel() for c in oracle.FDTD_COMPONENTS])
        got = np.concatenate([r.astype(np.float64).ravel() for r in result])
        return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
    return {"max_rel": float(np.max(np.abs(result.astype(np.float64) - full_ref) / np.abs(full_ref)))}


def bench_line(args, w, m, clk, world):
    """The contract's JSON line (without cpu_baseline and extras) from one
    workload's measurements `m` (measure_workload) and clock record `clk`.

    roofline.bound says what limits the workload: "hbm" when one step touches
    more than half of the L2 cache (the fields stream from DRAM every step),
    else "l2/latency" (the fields stay in L2; a launch's time is its load
    latency and the graph node's own cost, reported as per_node_us beside
    graph_node_floor_us, a node of the same launch shape doing almost no
    work).  achieved/frac are the in-step rate of algorithmic bytes against
    the measured HBM copy peak either way."""
    cells = cells_of(w)
    value, total_ms, _ = aggregate(m["graph_ms"], cells * w["iters"])
    ms_per_step = total_ms / args.steps
    per_step_value = cells * w["iters"] / (statistics.mean(m["per_step_ms"]) * 1e-3)
    peak, peak_kind = _peaks()
    bytes_launch = algo_bytes_per_launch(w, m["depth"], fused=m.get("fused", False))
    # average launch duration inside the timed region: CUDA events around
    # each graph-batched step on the launching stream, divided by the
    # kernel launches in it (so inter-node gaps are charged to the kernel)
    launch_ms = ms_per_step / m["launches"]
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    isolated = bytes_launch / (m["kern_ms"] * 1e-3) / 1e9
    ws = working_set_bytes(w)
    l2 = m.get("l2_bytes") or (126 << 20)
    bound = "hbm" if ws > 0.5 * l2 else "l2/latency"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(args.workload), "peak_kind": peak_kind,
            "working_set_bytes": ws, "l2_bytes": l2,
            "per_node_us": launch_ms * 1e3, "graph_node_floor_us": m.get("node_floor_us"),
            "launch_ms_in_step": launch_ms,
            "bytes_per_launch": bytes_launch, "isolated_launch_ms": m["kern_ms"],
            "isolated_GBps": isolated, "nominal_GBps": NOMINAL_HBM_GBS,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    if bound != "hbm":
        roof["note"] = ("working set in L2: frac compares the in-step rate of algorithmic bytes with the HBM copy "
                        "peak and is no HBM roofline; the HBM roofline of the same kernel is hbm_roofline")

    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step,
        "ms_per_step_std": statistics.pstdev(m["graph_ms"]) if len(m["graph_ms"]) > 1 else 0.0,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**config_of(args.workload, w, m["S"], m["depth"], world),
                   **({"tuned_plan": m["tuned_plan"]} if m.get("tuned_plan") else {"launch_plan": m.get("plan")})},
        "roofline": roof,
        "per_step_launch": {"value": per_step_value, "ms_per_step": statistics.mean(m["per_step_ms"]),
                            "ms_per_step_std": statistics.pstdev(m["per_step_ms"]) if len(m["per_step_ms"]) > 1 else 0.0,
                            "graph_speedup": (value / world) / per_step_value},
        "paper_convention": {"ms_build_plus_run": m["paper_conv_ms"], "build_s": m["build_s"]},
        "gpu_launches": m["launches"] * args.steps,
        "clocks": clk,
    }
    if m["e2e"] is not None:
        dt, h2d, d2h = m["e2e"]
        line["e2e"] = {"value": cells * w["iters"] / dt, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h}
    return line


def hbm_roofline_of(name, w, mm):
    """The HBM roofline figure of an HBM-bound workload's graph-batched run
    (measure_workload's record `mm`): in-step rate of algorithmic bytes per
    launch against the measured copy peak, with the cold-cache DRAM traffic
    and launch time of the committed ncu capture of the same kernel sources
    (None when the sources changed since)."""
    peak, peak_kind = _peaks()
    gms = statistics.mean(mm["graph_ms"])
    bl = algo_bytes_per_launch(w, mm["depth"])
    launch_ms = gms / mm["launches"]
    achieved = bl / (launch_ms * 1e-3) / 1e9
    traffic, cold_us = recorded_capture(name)
    out = {"workload": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic, "bytes_per_launch": bl,
           "per_launch_us_in_step": launch_ms * 1e3, "depth": mm["depth"], "S": mm["S"],
           "working_set_bytes": working_set_bytes(w)}
    if cold_us:
        out["cold_cache_us"] = cold_us
        out["cold_cache_frac"] = bl / (cold_us * 1e-6) / 1e9 / peak
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="iteration batch size S (0: workload default)")
    ap.add_argument("--depth", type=int, default=0, help="temporal depth t (0: workload default)")
    ap.add_argument("--block-x", type=int, default=0)
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--tile-x", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--pdl", action="store_true")
    ap.add_argument("--kernel", type=int, default=0, help="thermal kernel variant (gs_kernel; 0 = auto)")
    ap.add_argument("--loop", action="store_true",
                    help="run the batches as one device-side loop (conditional while node) per step")
    ap.add_argument("--traverse", type=int, default=0,
                    help="block order of consecutive launches (gs_traverse: 0 auto, 1 forward, 2 alternate)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the side measurements of the default run (other workloads, the batch-size sweep, "
                         "the 64-stream baseline, the FDTD storage-type errors)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle (timing and error checks)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = WORKLOADS[args.workload]

    if args.impl == "reference":
        run_reference(args, w, args.workload)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # All work (library, events, L2 flush) on one explicit stream: the
    # default stream's handle is 0, which the library reads as "create your
    # own stream", and events on another stream would not bracket its work.
    torch.cuda.set_stream(torch.cuda.Stream())
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2501_09398_gb300  # noqa: F401  (fails loudly without the CUDA library)

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(_smi_id())
    clocks.start()
    m = measure_workload(args.workload, w, args, flush)
    clk = clocks.stop()

    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    line = bench_line(args, w, m, clk, world)

    if rank == 0 and world == 1 and not args.no_cpu:
        v, sample, threads, full = oracle_sample(w)
        line["cpu_baseline"] = {"value": v, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
                                "sample": sample}
        line["cpu_baseline"]["single_thread"] = oracle_single_thread(w)
        err = error_vs_oracle(w, m["result"], full)
        if err is not None:
            line["error_vs_oracle"] = err
        if not args.no_extras and args.workload == DEFAULT:
            # the storage types' errors on the FDTD workload (one FP64 oracle run)
            try:
                line["fdtd_precision"] = fdtd_precision()
            except Exception as e:  # noqa: BLE001
                line["fdtd_precision"] = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0 and world == 1 and not args.no_extras and args.workload == DEFAULT:
        extra = {}
        peak = line["roofline"]["peak"]
        base = {**vars(args), "batch": 0, "depth": 0, "block_x": 0, "rows": 0, "tile_x": 0, "tile_y": 0,
                "pdl": False, "kernel": 0, "loop": False, "traverse": 0, "steps": 20}
        # 2D 512^2: graph-batched vs per-step launch of the same depth-1 kernel
        # 2D 4096^2: HBM roofline of the depth-1 kernel, and the wavefront
        # depth-4 kernel's throughput
        for nm, over, tag in (("heat2d-512", {}, "depth1"), ("heat2d-512", dict(loop=True), "device_loop"),
                              ("heat3d-256", {}, "column"),
                              ("heat3d-256", dict(depth=2, kernel=4, block_x=128), "zmarch2"),
                              ("heat3d-256", dict(depth=2, kernel=7, block_x=256), "stream2"),
                              ("fdtd-128", {}, "column"), ("fdtd-256", {}, "column"),
                              ("fdtd-128", dict(kernel=6, rows=4), "fused"), ("fdtd-256", dict(kernel=6, rows=8), "fused"),
                              ("fdtd-128", dict(kernel=6, rows=8, tile_y=8), "fused_march"),
                              ("fdtd-256", dict(kernel=6, rows=4, tile_y=8), "fused_march"),
                              ("fdtd-media-256", dict(kernel=6, rows=4, tile_y=8), "fused_march"),
                              ("fdtd-media-256", {}, "column"),
                              ("multi-64", {}, "tuned"),
                              ("heat2d-512", dict(depth=4, kernel=4, block_x=256), "column4"),
                              ("heat2d-4096", {}, "depth1"),
                              ("heat2d-4096", dict(depth=2, kernel=4, block_x=64), "column2"),
                              ("heat2d-4096", dict(depth=4, kernel=2, rows=32, block_x=128), "wave4")):
            ww = WORKLOADS[nm]
            mm = measure_workload(nm, ww, argparse.Namespace(**{**base, **over}), flush, with_e2e=False)
            c = cells_of(ww) * ww["iters"]
            gms = statistics.mean(mm["graph_ms"])
            gv = c / (gms * 1e-3)
            pv = c / (statistics.mean(mm["per_step_ms"]) * 1e-3)
            bl = algo_bytes_per_launch(ww, mm["depth"], fused=mm.get("fused", False))
            bw = bl / (gms / mm["launches"] * 1e-3) / 1e9
            extra[f"{nm}/{tag}"] = {"graph_value": gv, "per_step_value": pv, "graph_speedup": gv / pv,
                                    "S": mm["S"], "depth": mm["depth"], "in_step_GBps": bw,
                                    "hbm_frac": bw / peak, "paper_convention_ms": mm["paper_conv_ms"]}
            if mm.get("tuned_plan"):
                extra[f"{nm}/{tag}"]["tuned_plan"] = mm["tuned_plan"]
            if (nm, tag) == ("heat2d-4096", "depth1"):
                # the HBM roofline of the default workload's kernel (COLUMN,
                # depth 1) where the fields stream from DRAM every step
                line["hbm_roofline"] = hbm_roofline_of(nm, ww, mm)
        # the batch-size sweep of the 2D 512^2 and 3D 512x512x8 workloads at
        # temporal depths 1, 2 and 4; a failure here is recorded, not raised
        sweeps = {}
        for nm, plans in SWEEP_PLANS.items():
            try:
                sweeps[nm] = batch_sweep(WORKLOADS[nm], plans, flush)
            except Exception as e:  # noqa: BLE001
                sweeps[nm] = {"error": f"{type(e).__name__}: {e}"}
        extra["batch_sweep"] = sweeps
        # the instance batch's per-step baseline on 64 streams (the one-stream
        # baseline is multi-64/tuned's per_step_value)
        try:
            ms = multi_streams_per_step(WORKLOADS["multi-64"], flush)
            one = extra.get("multi-64/tuned", {})
            if one:
                ms["vs_one_stream_per_step"] = ms["value"] / one["per_step_value"]
                ms["fused_graph_speedup"] = one["graph_value"] / ms["value"]
            extra["multi-64/per_step_64_streams"] = ms
        except Exception as e:  # noqa: BLE001
            extra["multi-64/per_step_64_streams"] = {"error": f"{type(e).__name__}: {e}"}
        line["extra"] = extra

    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
