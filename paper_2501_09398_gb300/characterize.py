"""Characterise iteration batching on this GPU with the paper's skeleton
application (Sec. III-C, Sec. IV-A, Table I, Figs. 2-4 and 6).

For each workload size (1e3, 1e6, 1e7 elements, the paper's "threads"):

* creation: build time of a graph of S nodes (create + add nodes +
  instantiate + upload, ``gs_graph_build``) for S up to 2500, ten repetitions,
  fitted to Eq. 2 (T_C = k_c S + b_c);
* execution: device time of I_k = 10,000 iterations in graph batches of S
  (every divisor of I_k up to 2500, graphs already built), ten repetitions,
  fitted to Eq. 6 (T_E = a/S + b);
* the batch size minimising Eq. 1 over the divisors of I_k, and the relaxed
  optimum sqrt(a / k_c);
* device memory of an uploaded executable graph of S nodes (the drop in
  free memory across one build; the paper notes it grows linearly in S,
  Sec. IV-A);
* speed-up of graph batches of 100 over per-step launches for I = 1, 2, 3,
  5, 10, 100 batches, graph creation included (the paper's convention,
  Sec. IV-B).

Run ``python -m paper_2501_09398_gb300.characterize [--out file.json]``.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time

import numpy as np

from . import (GS_BC_CLAMP, GS_F32, GS_FIELD_X, GS_SKELETON, gs_bind_field, gs_create, gs_destroy, gs_get_stats,
               gs_graph_build, gs_graph_destroy, gs_model_fit, gs_model_pick, gs_set_scale, gs_step, gs_sync)

SIZES = (1_000, 1_000_000, 10_000_000)
I_K = 10_000
CREATE_S = (1, 10, 50, 100, 250, 500, 1000, 1500, 2000, 2500)


def _ctx(n, stream):
    import torch

    ctx = gs_create(GS_SKELETON, n, 1, 1, GS_F32, GS_BC_CLAMP, stream)
    buf = torch.ones(n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    gs_bind_field(ctx, GS_FIELD_X, buf.data_ptr(), n)
    gs_set_scale(ctx, 1.0)
    return ctx, buf


def _timed(ctx, stream, n_iters, S):
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    gs_step(ctx, n_iters, S)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) * 1e-3


def characterize(n, stream, reps=10):
    import torch

    ctx, keep = _ctx(n, stream.cuda_stream)
    try:
        gs_step(ctx, 200, 0)  # warm-up (module load, clocks)
        gs_sync(ctx)
        create, graph_mem = {}, {}
        for S in CREATE_S:
            ts = []
            for _ in range(reps):
                gs_graph_destroy(ctx)
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info()[0]
                gs_graph_build(ctx, S)
                graph_mem[S] = free0 - torch.cuda.mem_get_info()[0]
                ts.append(gs_get_stats(ctx)["last_build_seconds"])
            create[S] = ts
        divs = [d for d in range(1, 2501) if I_K % d == 0]
        execute = {}
        for S in divs:
            gs_graph_destroy(ctx)
            gs_graph_build(ctx, S)
            _timed(ctx, stream, I_K, S)  # warm
            execute[S] = [_timed(ctx, stream, I_K, S) for _ in range(reps)]
        mc = gs_model_fit(list(create), [statistics.mean(v) for v in create.values()],
                          [0.0] * len(create))
        me = gs_model_fit(list(execute), [0.0] * len(execute), [statistics.mean(v) for v in execute.values()])
        model = dict(k_c=mc["k_c"], b_c=mc["b_c"], a=me["a"], b=me["b"], mae_create=mc["mae_create"],
                     mae_exec=me["mae_exec"])
        best_S, best_T = gs_model_pick(model, divs)
        # measured optimum of T_C + T_E over the swept divisors
        meas = {S: statistics.mean(execute[S]) + (statistics.mean(create[S]) if S in create else
                                                 model["k_c"] * S + model["b_c"]) for S in divs}
        # speed-up of S = 100 batches vs per-step, creation included
        speed = {}
        for I in (1, 2, 3, 5, 10, 100):
            it = 100 * I
            base = [_timed(ctx, stream, it, 0) for _ in range(reps)]
            graph = []
            for _ in range(reps):
                gs_graph_destroy(ctx)
                t0 = time.perf_counter()
                gs_graph_build(ctx, 100)
                tc = time.perf_counter() - t0
                graph.append(tc + _timed(ctx, stream, it, 100))
            mb, mg = statistics.mean(base), statistics.mean(graph)
            err = (mb / mg) * math.sqrt((statistics.pstdev(base) / mb) ** 2 + (statistics.pstdev(graph) / mg) ** 2)
            speed[I] = dict(speedup=mb / mg, err=err)
        return dict(n=n, model=model, S_star_divisor=best_S, S_star_relaxed=math.sqrt(max(model["a"], 0) / model["k_c"]),
                    S_best_measured=min(meas, key=meas.get),
                    create_mean_s={S: statistics.mean(v) for S, v in create.items()},
                    graph_device_bytes=graph_mem,
                    exec_mean_s={S: statistics.mean(v) for S, v in execute.items()},
                    speedup_S100=speed)
    finally:
        gs_destroy(ctx)
        del keep


def main():
    import torch

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default="characterize.json")
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    res = [characterize(n, st, args.reps) for n in SIZES]
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    for r in res:
        m = r["model"]
        print(f"n={r['n']:>9}  k_c={m['k_c']:.3e} b_c={m['b_c']:.3e} MAE={m['mae_create']:.2e}  "
              f"a={m['a']:.3e} b={m['b']:.3e} MAE={m['mae_exec']:.2e}  S*={r['S_star_divisor']} "
              f"(relaxed {r['S_star_relaxed']:.0f}, measured {r['S_best_measured']})  "
              + " ".join(f"I={I}:{v['speedup']:.2f}" for I, v in r["speedup_S100"].items())
              + "  graph MiB: " + " ".join(f"S={S}:{b / 2**20:.1f}" for S, b in r["graph_device_bytes"].items()))


if __name__ == "__main__":
    main()
