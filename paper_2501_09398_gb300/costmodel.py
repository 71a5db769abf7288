"""Learned choice of iteration batch size, launch plan and temporal depth.

The paper picks the batch size S from a fitted analytic model (Sec. III-B,
Eqs. 1-6) and names automatic characterisation and selection as future work
(Sec. VI).  This module drives the library's own calls to do that with a
learned model:

1. ``sample_workloads``: seeded stepping problems over 2D 64^2-4096^2, 3D
   64^3-256^3 and thin 3D stacks, Yee FDTD 32^3-256^3, three storage types,
   run lengths I_k of 100-10000 iterations.
2. ``candidates``: per workload, the launch plans x batch sizes
   S in {per-step, 1, 10, 50, 100, 500, 1000}.
3. ``sweep``: times every candidate on the GPU with ``gs_autotune`` (graph
   build time T_C and milliseconds per iteration); the swept table is both
   the training data and the yardstick of every pick's regret.
4. ``train``: fits an ensemble of MLPs (``gs_mlp_*``: the library's CUDA
   forward, backward and Adam kernels; different seeds) to log(ms per
   iteration of the whole run), total = T_C + I_k * ms_per_iter; the pick
   minimises the members' mean prediction (``gs_mlp_argmin_ensemble``).
5. ``evaluate``: on held-out workloads, the regret of a pick is
   T(pick) / T(best in the sweep) - 1, for the learned picker, the paper's
   analytic picker (Eqs. 2 and 6 fitted to the same sweep at the default
   launch plan; reported with its calibration runs free and charged: it
   needs the workload's own timings at several batch sizes, the learned
   picker none) and a fixed S = 100 ("approximately 100 nodes", Sec. IV-A).

6. ``write_builtin``: the trained ensemble as the source file the library
   compiles in (``gs_mlp_create_builtin``, ``gs_pick_ctx``).
7. ``measured_regret``: the learned pick checked by running it: on held-out
   workloads, whole runs of I_k iterations (graph creation included, CUDA
   events on the stream) of the pick of the compiled-in ensemble, of the
   sweep's best candidate and of the analytic pick.

Run ``python -m paper_2501_09398_gb300.costmodel --help``.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import (GS_BC_CLAMP, GS_BC_PEC, GS_F32, GS_FDTD3D, GS_FIELD_P, GS_FIELD_T, GS_HEAT2D, GS_HEAT3D,
               GS_KERNEL_COLUMN, GS_MLP_INPUTS, FDTD_FIELDS, FdtdFields, HeatFields, gs_autotune, gs_create,
               gs_candidates, gs_destroy, gs_features, gs_graph_destroy, gs_model_fit, gs_model_pick,
               gs_mlp_argmin_ensemble, gs_mlp_create, gs_mlp_create_builtin, gs_mlp_destroy,
               gs_mlp_fit_normalization, gs_mlp_get_normalization, gs_mlp_get_params, gs_mlp_loss_grad,
               gs_mlp_train, gs_pick, gs_set_fdtd_params, gs_set_plan, gs_set_time, gs_step, gs_upload)

KINDS = ("heat2d", "heat3d", "fdtd")
KIND_ID = {"heat2d": GS_HEAT2D, "heat3d": GS_HEAT3D, "fdtd": GS_FDTD3D}


DATA = __import__("os").path.join(__import__("os").path.dirname(__file__), "data", "costmodel_sweep_gb300.json.gz")


def load_tables(path: str = DATA):
    """Swept (workload, table) pairs: the GB300 sweep shipped with the
    package (150 training workloads, seed 1; 200 held-out, seed 4242), or a
    file written by --dataset.  Returns (train_pairs, heldout_pairs)."""
    import gzip

    opener = gzip.open if path.endswith(".gz") else open
    with opener(path, "rt") as f:
        d = json.load(f)
    for split in ("train", "heldout"):
        for _, tab in d[split]:
            for r in tab:
                if r["ms_per_iter"] is None:
                    r["ms_per_iter"] = float("inf")
    return [tuple(p) for p in d["train"]], [tuple(p) for p in d["heldout"]]


def sample_workloads(n: int, seed: int):
    """n seeded workloads (dicts with kind, dtype, nx, ny, nz, n_iters)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        kind = KINDS[int(rng.integers(0, 3))]
        dtype = int(rng.integers(0, 3))
        n_iters = int(round(math.exp(rng.uniform(math.log(100), math.log(10000)))))
        lu = lambda lo, hi: int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))  # noqa: E731
        if kind == "heat2d":
            nx, ny, nz = lu(64, 4096), lu(64, 4096), 1
        elif kind == "heat3d":
            if rng.uniform() < 0.5:
                nx, ny, nz = lu(64, 256), lu(64, 256), lu(64, 256)
            else:  # thin stack (Hotspot3D-like chips): few layers, wide planes
                nx, ny, nz = lu(128, 1024), lu(128, 1024), int(rng.choice([2, 4, 8, 16]))
        else:
            nx = ny = nz = lu(32, 256)
        out.append(dict(kind=kind, dtype=dtype, nx=nx, ny=ny, nz=nz, n_iters=n_iters))
    return out


def default_plan(w):
    """The library's default launch plan for the workload (what gs_create
    picks), used by the analytic and fixed pickers."""
    if w["kind"] == "fdtd":
        return dict(block_x=64, rows=4, temporal_depth=1, kernel=GS_KERNEL_COLUMN, tile_y=0)
    small = w["nx"] * w["ny"] * w["nz"] <= (1 << 22)
    deep = w["kind"] == "heat3d" and w["nz"] > 8
    return dict(block_x=64, rows=4 if (small or deep) else 8, temporal_depth=1, kernel=GS_KERNEL_COLUMN, tile_y=0)


def candidates(w):
    """(plan, S) pairs for a workload, plan after plan, as the library lists
    them (gs_candidates): block_x, rows, temporal_depth and kernel explicit."""
    return gs_candidates(_fw(w))


def _context(w, stream):
    """A context for the workload with seeded fields; returns (ctx, keepalive)."""
    import gs_inputs

    kind = KIND_ID[w["kind"]]
    if w["kind"] == "fdtd":
        N = w["nx"]
        ctx = gs_create(kind, N, N, N, w["dtype"], GS_BC_PEC, stream)
        f = FdtdFields(ctx, N, w["dtype"])
        gs_set_fdtd_params(ctx, courant=0.5, src_on=1, src=(N // 2, N // 2, N // 2))
        return ctx, f
    ctx = gs_create(kind, w["nx"], w["ny"], w["nz"], w["dtype"], GS_BC_CLAMP, stream)
    f = HeatFields(ctx, w["nx"], w["ny"], w["nz"], w["dtype"])
    T, P = gs_inputs.heat_fields(w["nx"], w["ny"], w["nz"], seed=0)
    gs_upload(ctx, GS_FIELD_T, T)
    gs_upload(ctx, GS_FIELD_P, P)
    return ctx, f


def sweep(w, n_meas: int = 1000, reps: int = 1, stream=None):
    """Time every candidate of w; returns a list of dicts (plan, S,
    build_seconds, ms_per_iter, status)."""
    ctx, keep = _context(w, stream)
    try:
        cands = candidates(w)
        res, _ = gs_autotune(ctx, n_meas, cands, reps=reps)
    finally:
        gs_destroy(ctx)
        del keep
    out = []
    for (plan, S), r in zip(cands, res):
        out.append(dict(plan=plan, S=S, build_seconds=r["build_seconds"], ms_per_iter=r["exec_ms_per_iter"],
                        status=r["status"]))
    return out


def run_ms(row, n_iters):
    """Modelled wall time of an n_iters run of a swept candidate:
    graph creation plus n_iters steady-state iterations."""
    return row["build_seconds"] * 1e3 + n_iters * row["ms_per_iter"]


def _fw(w):
    """The workload as gs_features takes it (numeric kind)."""
    return dict(w, kind=KIND_ID[w["kind"]])


def rows_for(w, table, n_iters_list=None):
    """Training rows (features, log ms per iteration) of a swept workload."""
    ok = [r for r in table if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
    feats, ys = [], []
    for n in (n_iters_list or [w["n_iters"]]):
        F = gs_features(_fw(dict(w, n_iters=n)), [(r["plan"], r["S"]) for r in ok])
        feats.append(F)
        ys.append(np.array([math.log(run_ms(r, n) / n) for r in ok], dtype=np.float32))
    return np.concatenate(feats), np.concatenate(ys)


# Run lengths each swept workload contributes rows for (besides its own):
# the table gives T_C and ms per iteration, so any run length can be
# composed; spreading them teaches the model how T_C amortises.
AUG_ITERS = tuple(int(v) for v in np.geomspace(100, 10000, 7))


def training_set(pairs):
    """Stack the training rows of (workload, table) pairs."""
    Xs, ys = [], []
    for w, tab in pairs:
        X, y = rows_for(w, tab, [w["n_iters"], *AUG_ITERS])
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


# Members of the model ensemble.  Single networks trained from different
# seeds land 3-6 % mean regret apart on the held-out workloads; the mean
# prediction of three is steadier (about 3 %).
ENSEMBLE = 3


def train(X: np.ndarray, y: np.ndarray, epochs: int = 2000, batch_rows: int = 1024, lr: float = 1e-3, seed: int = 0,
          stream=None, members: int = ENSEMBLE):
    """Fit `members` MLPs (seeds seed, seed+1, ...) on device copies of
    (X, y); returns (list of model handles, initial losses, final losses)."""
    import torch

    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    torch.cuda.synchronize()
    models, l0s, losses = [], [], []
    try:
        for k in range(members):
            m = gs_mlp_create(seed=seed + k, stream=stream)
            models.append(m)
            gs_mlp_fit_normalization(m, Xd.data_ptr(), X.shape[0])
            l0, _ = gs_mlp_loss_grad(m, Xd.data_ptr(), yd.data_ptr(), X.shape[0])
            l0s.append(l0)
            losses.append(gs_mlp_train(m, Xd.data_ptr(), yd.data_ptr(), X.shape[0], epochs, batch_rows, lr))
    except Exception:
        for m in models:
            gs_mlp_destroy(m)
        raise
    return models, l0s, losses


def pick_learned(models, w, table):
    """The swept candidate the ensemble predicts fastest (among runnable ones)."""
    import torch

    ok = [r for r in table if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
    F = gs_features(_fw(w), [(r["plan"], r["S"]) for r in ok])
    Fd = torch.from_numpy(F).cuda()
    torch.cuda.synchronize()
    idx, _ = gs_mlp_argmin_ensemble(models, Fd.data_ptr(), F.shape[0])
    return ok[idx]


def pick_analytic(w, table):
    """The paper's method: at the default launch plan, fit Eq. 2 to the
    measured build times and Eq. 6 to the measured execution times of the
    graph batch sizes, then take the S minimising Eq. 1 for I_k = n_iters."""
    dp = default_plan(w)
    rows = [r for r in table if r["plan"] == dp and r["S"] > 0 and r["status"] == 0]
    S = [r["S"] for r in rows]
    tc = [r["build_seconds"] for r in rows]
    te = [w["n_iters"] * r["ms_per_iter"] * 1e-3 for r in rows]
    model = gs_model_fit(S, tc, te)
    best, _ = gs_model_pick(model, S)
    return next(r for r in rows if r["S"] == best)


def pick_fixed(w, table, S=100):
    dp = default_plan(w)
    return next(r for r in table if r["plan"] == dp and r["S"] == S and r["status"] == 0)


def calibration_ms(w, table):
    """The least the analytic picker must spend on a new workload before it
    can pick: one graph build and one launch of every batch size it fits
    Eqs. 2 and 6 to, at the default plan (the learned picker runs nothing)."""
    dp = default_plan(w)
    rows = [r for r in table if r["plan"] == dp and r["S"] > 0 and r["status"] == 0]
    return sum(r["build_seconds"] * 1e3 + r["S"] * r["ms_per_iter"] for r in rows)


def regret(w, table, row):
    ok = [r for r in table if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
    best = min(run_ms(r, w["n_iters"]) for r in ok)
    return run_ms(row, w["n_iters"]) / best - 1.0


def evaluate(models, held):
    """held: list of (workload, table).  Returns per-picker regrets; the
    analytic picker's twice: with its calibration runs free (fitted on the
    workload's own swept timings) and with them charged to the run."""
    out = {"learned": [], "analytic": [], "analytic_with_calibration": [], "fixed_S100": []}
    for w, table in held:
        out["learned"].append(regret(w, table, pick_learned(models, w, table)))
        ra = regret(w, table, pick_analytic(w, table))
        out["analytic"].append(ra)
        ok = [r for r in table if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
        best = min(run_ms(r, w["n_iters"]) for r in ok)
        out["analytic_with_calibration"].append(ra + calibration_ms(w, table) / best)
        out["fixed_S100"].append(regret(w, table, pick_fixed(w, table)))
    return out


def summarize(reg):
    return {k: dict(mean=float(np.mean(v)), median=float(np.median(v)), p95=float(np.percentile(v, 95)),
                    max=float(np.max(v)), within_5pct=float(np.mean(np.array(v) <= 0.05))) for k, v in reg.items()}


BUILTIN = __import__("os").path.join(__import__("os").path.dirname(__file__), "csrc", "costmodel_weights.inc")


def write_builtin(models, path: str, info: str) -> None:
    """Write the ensemble's parameters and normalisation as the C++ include
    the library compiles in (exact float32 values, 9 significant digits)."""
    def arr(v):
        return ",".join("%.9g" % float(x) for x in v)

    params = [gs_mlp_get_params(m) for m in models]
    norms = [np.concatenate(gs_mlp_get_normalization(m)) for m in models]
    lines = ["// The cost-model ensemble compiled into the library (see mlp.cu,",
             "// gs_mlp_create_builtin), written by",
             "// `python -m paper_2501_09398_gb300.costmodel --write-builtin FILE`.",
             "constexpr int kBuiltinTrained = 1;",
             "constexpr int kBuiltinMembers = %d;" % len(models),
             "static const float kBuiltinParams[kBuiltinMembers][GS_MLP_PARAMS] = {"]
    lines += ["    {%s}," % arr(p) for p in params]
    lines += ["};", "static const float kBuiltinNorm[kBuiltinMembers][2 * GS_MLP_INPUTS] = {"]
    lines += ["    {%s}," % arr(n) for n in norms]
    lines += ["};", "static const char kBuiltinInfo[] = %s;" % json.dumps(info)]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def builtin_models(stream=None):
    return [gs_mlp_create_builtin(k, stream) for k in range(3)]


def _reset(ctx, w):
    """Seeded initial state of the workload's fields (outside any timing)."""
    import gs_inputs

    if w["kind"] == "fdtd":
        z = np.zeros((w["nx"] + 1,) * 3, dtype=np.float32)
        for fid in FDTD_FIELDS:
            gs_upload(ctx, fid, z)
        gs_set_time(ctx, 0)
    else:
        T, P = gs_inputs.heat_fields(w["nx"], w["ny"], w["nz"], seed=0)
        gs_upload(ctx, GS_FIELD_T, T)
        gs_upload(ctx, GS_FIELD_P, P)


def whole_run_ms(w, plan, S, stream, reps=3):
    """Median over `reps` runs (after one untimed run) of a whole run of
    w["n_iters"] iterations with (plan, S) from a fresh state: graph
    creation (T_C) and execution, CUDA events on the context's stream (the
    GPU waits for the host's graph build between them).  `stream`: a CUDA
    stream handle (not NULL), the context's and the events'."""
    import torch

    assert stream, "whole_run_ms needs the stream its context and events share"

    ctx, keep = _context(w, stream)
    try:
        gs_set_plan(ctx, **plan)
        st = torch.cuda.ExternalStream(stream)  # the context's stream
        times = []
        for r in range(reps + 1):
            _reset(ctx, w)
            gs_graph_destroy(ctx)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            gs_step(ctx, w["n_iters"], S)
            b.record(st)
            torch.cuda.synchronize()
            if r > 0:
                times.append(a.elapsed_time(b))
    finally:
        gs_destroy(ctx)
        del keep
    return float(np.median(times))


def measured_regret(models, held, n=30, seed=7, stream=None, reps=3, max_run_ms=400.0):
    """Whole-run regret of the learned pick, measured: for n held-out
    workloads (a seeded choice, equal numbers of each kind, runs the sweep
    predicts under max_run_ms), run the learned pick (gs_pick with
    `models`), the sweep's best candidate and the analytic pick, each a
    whole run of I_k iterations; regret = T(pick) / min over the three - 1.
    Returns per-workload records and the composed-time regrets (from the
    sweep's T_C and ms per iteration) of the same picks."""
    import torch

    if stream is None:  # the contexts and the timing events must share one stream
        stream = torch.cuda.Stream().cuda_stream
    rng = np.random.default_rng(seed)
    by_kind = {k: [] for k in KINDS}
    for w, tab in held:
        ok = [r for r in tab if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
        if ok and min(run_ms(r, w["n_iters"]) for r in ok) < max_run_ms:
            by_kind[w["kind"]].append((w, tab))
    chosen = []
    for k in KINDS:
        idx = rng.permutation(len(by_kind[k]))[: n // len(KINDS)]
        chosen += [by_kind[k][i] for i in sorted(idx)]
    recs = []
    for w, tab in chosen:
        plan_l, S_l, _ = gs_pick(models, _fw(w))
        ok = [r for r in tab if r["status"] == 0 and math.isfinite(r["ms_per_iter"])]
        best = min(ok, key=lambda r: run_ms(r, w["n_iters"]))
        ana = pick_analytic(w, tab)
        picks = {"learned": (plan_l, S_l), "swept_best": (best["plan"], best["S"]), "analytic": (ana["plan"], ana["S"])}
        meas = {}
        for name, (plan, S) in picks.items():
            key = (tuple(sorted(plan.items())), S)
            same = [m for m in meas.values() if m["key"] == key]
            meas[name] = dict(key=key, ms=same[0]["ms"] if same else whole_run_ms(w, plan, S, stream, reps))
        lo = min(m["ms"] for m in meas.values())
        learned_row = next((r for r in ok if r["plan"] == plan_l and r["S"] == S_l), None)
        recs.append(dict(workload=w, ms={k: v["ms"] for k, v in meas.items()},
                         measured_regret={k: v["ms"] / lo - 1.0 for k, v in meas.items()},
                         composed_regret_learned=(regret(w, tab, learned_row) if learned_row else None),
                         picks={k: dict(plan=v[0], S=v[1]) for k, v in picks.items()}))
    return recs


def summarize_measured(recs):
    out = {}
    for name in ("learned", "swept_best", "analytic"):
        v = np.array([r["measured_regret"][name] for r in recs])
        out[name] = dict(mean=float(v.mean()), median=float(np.median(v)), p95=float(np.percentile(v, 95)),
                         within_5pct=float(np.mean(v <= 0.05)))
    comp = [r["composed_regret_learned"] for r in recs if r["composed_regret_learned"] is not None]
    out["learned_composed_same_workloads"] = dict(mean=float(np.mean(comp)), n=len(comp))
    out["workloads"] = len(recs)
    return out


def main():
    import torch

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", type=int, default=150, help="training workloads (seed 1)")
    ap.add_argument("--heldout", type=int, default=200, help="held-out workloads (seed 4242)")
    ap.add_argument("--n-meas", type=int, default=1000, help="iterations per timed run in the sweep")
    ap.add_argument("--epochs", type=int, default=2000)
    ap.add_argument("--out", default="costmodel_report.json")
    ap.add_argument("--dataset", default="", help="write the swept tables here (json)")
    ap.add_argument("--tables", default="",
                    help="read swept tables instead of sweeping: a --dataset file, or 'packaged' for the GB300 sweep")
    ap.add_argument("--batch-rows", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--members", type=int, default=ENSEMBLE, help="models in the ensemble")
    ap.add_argument("--write-builtin", default="",
                    help="write the trained ensemble as the include the library compiles in (e.g. " + BUILTIN + ")")
    ap.add_argument("--measure-regret", type=int, default=0,
                    help="only measure whole-run regret of the compiled-in ensemble on this many held-out workloads "
                         "(--tables gives the sweep)")
    ap.add_argument("--regret-seed", type=int, default=7, help="seed of the workload choice of --measure-regret")
    ap.add_argument("--regret-max-ms", type=float, default=400.0,
                    help="--measure-regret takes workloads whose swept best run is shorter than this")
    ap.add_argument("--regret-reps", type=int, default=3, help="timed runs per pick (median)")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    t0 = time.time()
    if args.measure_regret:
        _, held_pairs = load_tables(DATA if args.tables in ("", "packaged") else args.tables)
        models = builtin_models(st.cuda_stream)
        try:
            recs = measured_regret(models, held_pairs, n=args.measure_regret, seed=args.regret_seed,
                                   stream=st.cuda_stream, reps=args.regret_reps, max_run_ms=args.regret_max_ms)
        finally:
            for m in models:
                gs_mlp_destroy(m)
        report = dict(summary=summarize_measured(recs), records=recs, seconds=time.time() - t0)
        with open(args.out, "w") as f:
            json.dump(report, f, indent=1, default=str)
        print(json.dumps(report["summary"]))
        return
    if args.tables:
        train_pairs, held_pairs = load_tables(DATA if args.tables == "packaged" else args.tables)
        train_pairs, held_pairs = train_pairs[:args.train], held_pairs[:args.heldout]
    else:
        train_w = sample_workloads(args.train, seed=1)
        held_w = sample_workloads(args.heldout, seed=4242)
        train_pairs = [(w, sweep(w, args.n_meas, stream=st.cuda_stream)) for w in train_w]
        held_pairs = [(w, sweep(w, args.n_meas, stream=st.cuda_stream)) for w in held_w]
        if args.dataset:
            with open(args.dataset, "w") as f:
                json.dump(dict(train=train_pairs, heldout=held_pairs), f)
    t_sweep = time.time() - t0
    X, y = training_set(train_pairs)
    models, l0, loss = train(X, y, epochs=args.epochs, batch_rows=args.batch_rows, lr=args.lr, members=args.members)
    try:
        reg = evaluate(models, held_pairs)
        if args.write_builtin:
            info = ("GB300 ensemble of %d MLPs (seeds 0..%d), %d epochs, batch %d, lr %g, trained on %d rows from %d "
                    "swept workloads (seed 1); final losses %s; held-out mean regret %.4f (composed from the sweep)"
                    % (len(models), len(models) - 1, args.epochs, args.batch_rows, args.lr, X.shape[0],
                       len(train_pairs), ", ".join("%.4f" % v for v in loss), float(np.mean(reg["learned"]))))
            write_builtin(models, args.write_builtin, info)
    finally:
        for m in models:
            gs_mlp_destroy(m)
    report = dict(train_workloads=len(train_pairs), heldout_workloads=len(held_pairs), rows=int(X.shape[0]),
                  epochs=args.epochs, batch_rows=args.batch_rows, lr=args.lr, members=args.members,
                  loss_initial=l0, loss_final=loss, sweep_seconds=t_sweep, regret=summarize(reg))
    with open(args.out, "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report))


if __name__ == "__main__":
    main()
