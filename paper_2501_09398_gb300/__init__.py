"""Python binding of libgraphstep (C ABI declared in include/graphstep.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, converts Python/NumPy/PyTorch arguments to pointers and
sizes, and raises ``GsError`` when the call returns a status other than
GS_OK.  All stepping runs in the library's CUDA kernels; there is no CPU
fallback, and importing this package fails if libgraphstep.so is missing
(build it with ``python paper_2501_09398_gb300/build.py``).

PyTorch is used only as a source of device memory and streams: pass
``tensor.data_ptr()`` / ``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GS_LIBRARY=checked loads the bounds-checked test build instead
LIB_PATH = os.path.join(_HERE, "libgraphstep_checked.so" if os.environ.get("GS_LIBRARY") == "checked"
                        else "libgraphstep.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} not found: the CUDA library must be built first "
        "(python paper_2501_09398_gb300/build.py)")

_lib = ctypes.CDLL(LIB_PATH)

# ------------------------------------------------------------ constants --
GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_STATE, GS_ERR_TIMEOUT, GS_ERR_NUMERIC, \
    GS_ERR_UNSUPPORTED = range(8)
GS_HEAT2D, GS_HEAT3D, GS_FDTD3D, GS_SKELETON = range(4)
GS_F32, GS_BF16, GS_F16 = range(3)
GS_BC_CLAMP, GS_BC_DIRICHLET0, GS_BC_PEC = range(3)
GS_KERNEL_AUTO, GS_KERNEL_MARCH, GS_KERNEL_WAVE, GS_KERNEL_TILE, GS_KERNEL_COLUMN, GS_KERNEL_COLUMN_SMEM, \
    GS_KERNEL_FUSED, GS_KERNEL_STREAM = range(8)
GS_TRAVERSE_AUTO, GS_TRAVERSE_FORWARD, GS_TRAVERSE_ALTERNATE = range(3)
(GS_FIELD_T0, GS_FIELD_T1, GS_FIELD_P, GS_FIELD_EX, GS_FIELD_EY, GS_FIELD_EZ, GS_FIELD_HX, GS_FIELD_HY,
 GS_FIELD_HZ, GS_FIELD_T, GS_FIELD_X, GS_FIELD_MAT) = range(12)
GS_MAX_MEDIA = 256

DTYPES = {"f32": GS_F32, "bf16": GS_BF16, "f16": GS_F16}
FDTD_FIELDS = (GS_FIELD_EX, GS_FIELD_EY, GS_FIELD_EZ, GS_FIELD_HX, GS_FIELD_HY, GS_FIELD_HZ)


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.gs_status_string(status).decode()}: {msg}")
        self.status = status


# ---------------------------------------------------------------- structs --
class gs_heat_coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("k", "cx", "cy", "cz", "cz2", "t_amb")]


class gs_fdtd_params(ctypes.Structure):
    _fields_ = [("courant", ctypes.c_float), ("src_on", ctypes.c_int32), ("src_i", ctypes.c_int64),
                ("src_j", ctypes.c_int64), ("src_k", ctypes.c_int64), ("src_amp", ctypes.c_float),
                ("src_delay", ctypes.c_float), ("src_width", ctypes.c_float)]


class gs_medium(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("eps_r", "sigma", "mu_r", "sigma_m")]


class gs_plan(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("block_x", "rows", "tile_x", "tile_y", "temporal_depth", "use_pdl",
                                              "device_launch", "kernel", "graph_loop", "traverse")]


class gs_multi_plan(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("block_x", "rows", "blocks", "use_pdl", "kernel", "traverse",
                                              "temporal_depth")]


class gs_tune_candidate(ctypes.Structure):
    _fields_ = [("plan", gs_plan), ("batch_size", ctypes.c_int64)]


class gs_tune_result(ctypes.Structure):
    _fields_ = [("plan", gs_plan), ("batch_size", ctypes.c_int64), ("build_seconds", ctypes.c_double),
                ("exec_ms_per_iter", ctypes.c_double), ("total_ms", ctypes.c_double), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class gs_model(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("k_c", "b_c", "a", "b", "mae_create", "mae_exec")]


class gs_stats(ctypes.Structure):
    _fields_ = [("last_build_seconds", ctypes.c_double), ("last_build_nodes", ctypes.c_int64),
                ("graphs_built", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("iterations", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_fp = ctypes.POINTER(ctypes.c_float)


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("gs_version", [])
_sig("gs_status_string", [ctypes.c_int], ctypes.c_char_p)
_sig("gs_last_error", [_vp], ctypes.c_char_p)
_sig("gs_required_pitch", [ctypes.c_int, _i64, ctypes.POINTER(_i64)])
_sig("gs_create", [ctypes.POINTER(_vp), ctypes.c_int, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int, _vp])
_sig("gs_destroy", [_vp])
_sig("gs_set_heat_coeffs", [_vp, ctypes.POINTER(gs_heat_coeffs)])
_sig("gs_set_fdtd_params", [_vp, ctypes.POINTER(gs_fdtd_params)])
_sig("gs_set_fdtd_media", [_vp, ctypes.POINTER(gs_medium), ctypes.c_int32])
_sig("gs_upload_u8", [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8), _i64])
_sig("gs_set_plan", [_vp, ctypes.POINTER(gs_plan)])
_sig("gs_set_scale", [_vp, ctypes.c_float])
_sig("gs_get_plan", [_vp, ctypes.POINTER(gs_plan)])
_sig("gs_bind_field", [_vp, ctypes.c_int, _vp, _i64])
_sig("gs_upload", [_vp, ctypes.c_int, _fp, _i64])
_sig("gs_read_field", [_vp, ctypes.c_int, _fp, _i64])
_sig("gs_get_parity", [_vp, ctypes.POINTER(_i32)])
_sig("gs_set_parity", [_vp, _i32])
_sig("gs_set_time", [_vp, _i64])
_sig("gs_get_time", [_vp, ctypes.POINTER(_i64)])
_sig("gs_step", [_vp, _i64, _i64])
_sig("gs_graph_build", [_vp, _i64])
_sig("gs_graph_launch", [_vp, _i64])
_sig("gs_graph_destroy", [_vp])
_sig("gs_sync", [_vp])
_sig("gs_get_stats", [_vp, ctypes.POINTER(gs_stats)])
_i64p = ctypes.POINTER(_i64)
_sig("gs_autotune", [_vp, _i64, _i32, ctypes.POINTER(gs_tune_candidate), _i32, ctypes.POINTER(gs_tune_result),
                     ctypes.POINTER(_i32)])
_sig("gs_multi_create", [ctypes.POINTER(_vp), _i32, _i64p, _i64p, ctypes.c_int, ctypes.c_int, _vp])
_sig("gs_multi_destroy", [_vp])
_sig("gs_multi_last_error", [_vp], ctypes.c_char_p)
_sig("gs_multi_set_heat_coeffs", [_vp, ctypes.POINTER(gs_heat_coeffs)])
_sig("gs_multi_set_plan", [_vp, ctypes.POINTER(gs_multi_plan)])
_sig("gs_multi_bind_field", [_vp, _i32, ctypes.c_int, _vp, _i64])
_sig("gs_multi_upload", [_vp, _i32, ctypes.c_int, _fp, _i64])
_sig("gs_multi_read_field", [_vp, _i32, ctypes.c_int, _fp, _i64])
_sig("gs_multi_step", [_vp, _i64, _i64, ctypes.c_int])
_sig("gs_multi_get_parity", [_vp, ctypes.POINTER(_i32)])
_sig("gs_multi_sync", [_vp])
_sig("gs_multi_get_stats", [_vp, ctypes.POINTER(gs_stats)])


def _check(st: int, ctx=None):
    if st != GS_OK:
        raise GsError(st, _lib.gs_last_error(ctx).decode(errors="replace"))


def _f32_ptr(a: np.ndarray):
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("need a C-contiguous float32 array")
    return a.ctypes.data_as(_fp)


# --------------------------------------------------------------- calls -----
def gs_version() -> int:
    return int(_lib.gs_version())


def gs_status_string(status: int) -> str:
    return _lib.gs_status_string(status).decode()


def gs_last_error(ctx) -> str:
    return _lib.gs_last_error(ctx).decode(errors="replace")


def gs_required_pitch(dtype: int, width: int) -> int:
    out = _i64()
    _check(_lib.gs_required_pitch(dtype, width, ctypes.byref(out)))
    return out.value


def gs_create(kind: int, nx: int, ny: int, nz: int, dtype: int = GS_F32, bc: int = GS_BC_CLAMP, stream=None):
    """Return an opaque context handle (ctypes.c_void_p)."""
    h = _vp()
    _check(_lib.gs_create(ctypes.byref(h), kind, nx, ny, nz, dtype, bc, _vp(stream) if stream else None))
    return h


def gs_destroy(ctx) -> None:
    _check(_lib.gs_destroy(ctx))


def gs_set_heat_coeffs(ctx, k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.05, t_amb=80.0) -> None:
    c = gs_heat_coeffs(k, cx, cy, cz, cz2, t_amb)
    _check(_lib.gs_set_heat_coeffs(ctx, ctypes.byref(c)), ctx)


def gs_set_fdtd_params(ctx, courant=0.5, src_on=0, src=(0, 0, 0), amp=1.0, delay=60.0, width=20.0) -> None:
    p = gs_fdtd_params(courant, src_on, src[0], src[1], src[2], amp, delay, width)
    _check(_lib.gs_set_fdtd_params(ctx, ctypes.byref(p)), ctx)


def gs_set_scale(ctx, c: float) -> None:
    _check(_lib.gs_set_scale(ctx, c), ctx)


def gs_set_plan(ctx, block_x=0, rows=0, tile_x=0, tile_y=0, temporal_depth=0, use_pdl=0, device_launch=0,
                kernel=0, graph_loop=0, traverse=0) -> None:
    p = gs_plan(block_x, rows, tile_x, tile_y, temporal_depth, use_pdl, device_launch, kernel, graph_loop, traverse)
    _check(_lib.gs_set_plan(ctx, ctypes.byref(p)), ctx)


def gs_get_plan(ctx) -> dict:
    p = gs_plan()
    _check(_lib.gs_get_plan(ctx, ctypes.byref(p)), ctx)
    return {n: getattr(p, n) for n, _ in gs_plan._fields_}


def gs_bind_field(ctx, field: int, ptr: int, pitch: int) -> None:
    _check(_lib.gs_bind_field(ctx, field, _vp(ptr) if ptr else None, pitch), ctx)


def gs_upload(ctx, field: int, host: np.ndarray) -> None:
    _check(_lib.gs_upload(ctx, field, _f32_ptr(host), host.size), ctx)


def gs_upload_u8(ctx, field: int, host: np.ndarray) -> None:
    host = np.ascontiguousarray(host, dtype=np.uint8)
    _check(_lib.gs_upload_u8(ctx, field, host.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), host.size), ctx)


def gs_set_fdtd_media(ctx, table) -> None:
    """table: rows of (eps_r, sigma, mu_r, sigma_m); empty for vacuum."""
    rows = list(table)
    arr = (gs_medium * max(1, len(rows)))(*[gs_medium(*map(float, r)) for r in rows])
    _check(_lib.gs_set_fdtd_media(ctx, arr, len(rows)), ctx)


def gs_read_field(ctx, field: int, out: np.ndarray) -> np.ndarray:
    _check(_lib.gs_read_field(ctx, field, _f32_ptr(out), out.size), ctx)
    return out


def gs_get_parity(ctx) -> int:
    v = _i32()
    _check(_lib.gs_get_parity(ctx, ctypes.byref(v)), ctx)
    return v.value


def gs_set_parity(ctx, parity: int) -> None:
    _check(_lib.gs_set_parity(ctx, parity), ctx)


def gs_set_time(ctx, n: int) -> None:
    _check(_lib.gs_set_time(ctx, n), ctx)


def gs_get_time(ctx) -> int:
    v = _i64()
    _check(_lib.gs_get_time(ctx, ctypes.byref(v)), ctx)
    return v.value


def gs_step(ctx, n_iters: int, batch_size: int) -> None:
    _check(_lib.gs_step(ctx, n_iters, batch_size), ctx)


def gs_graph_build(ctx, batch_size: int) -> None:
    _check(_lib.gs_graph_build(ctx, batch_size), ctx)


def gs_graph_launch(ctx, n_launches: int) -> None:
    _check(_lib.gs_graph_launch(ctx, n_launches), ctx)


def gs_graph_destroy(ctx) -> None:
    _check(_lib.gs_graph_destroy(ctx), ctx)


def gs_sync(ctx) -> None:
    _check(_lib.gs_sync(ctx), ctx)


def gs_get_stats(ctx) -> dict:
    s = gs_stats()
    _check(_lib.gs_get_stats(ctx, ctypes.byref(s)), ctx)
    return {n: getattr(s, n) for n, _ in gs_stats._fields_}


def _plan_dict(p) -> dict:
    return {n: getattr(p, n) for n, _ in gs_plan._fields_}


def gs_autotune(ctx, n_iters: int, candidates, reps: int = 3):
    """candidates: list of (plan dict, batch_size).  Returns (results, best
    index); each result is a dict with the plan as applied, batch_size,
    build_seconds, exec_ms_per_iter, total_ms and status."""
    n = len(candidates)
    arr = (gs_tune_candidate * n)()
    for i, (plan, S) in enumerate(candidates):
        arr[i].plan = gs_plan(*[int(plan.get(f, 0)) for f, _ in gs_plan._fields_])
        arr[i].batch_size = int(S)
    res = (gs_tune_result * n)()
    best = _i32(-1)
    _check(_lib.gs_autotune(ctx, n_iters, reps, arr, n, res, ctypes.byref(best)), ctx)
    out = [dict(plan=_plan_dict(r.plan), batch_size=r.batch_size, build_seconds=r.build_seconds,
                exec_ms_per_iter=r.exec_ms_per_iter, total_ms=r.total_ms, status=r.status) for r in res]
    return out, best.value


_dp = ctypes.POINTER(ctypes.c_double)
_sig("gs_model_fit", [_dp, _dp, _dp, _i32, ctypes.POINTER(gs_model)])
_sig("gs_model_total", [ctypes.POINTER(gs_model), ctypes.c_double, _dp])
_sig("gs_model_pick", [ctypes.POINTER(gs_model), ctypes.POINTER(_i64), _i32, ctypes.POINTER(_i64), _dp])
_sig("gs_model_calibrate", [_vp, _i64, ctypes.POINTER(_i64), _i32, _i32, ctypes.POINTER(gs_model)])


def _model_dict(m) -> dict:
    return {n: getattr(m, n) for n, _ in gs_model._fields_}


def _model_struct(d) -> "gs_model":
    return gs_model(*[float(d.get(n, 0.0)) for n, _ in gs_model._fields_])


def gs_model_fit(S, t_create, t_exec) -> dict:
    n = len(S)
    arr = lambda v: (ctypes.c_double * n)(*[float(x) for x in v])  # noqa: E731
    out = gs_model()
    _check(_lib.gs_model_fit(arr(S), arr(t_create), arr(t_exec), n, ctypes.byref(out)))
    return _model_dict(out)


def gs_model_total(model: dict, S: float) -> float:
    out = ctypes.c_double()
    _check(_lib.gs_model_total(ctypes.byref(_model_struct(model)), float(S), ctypes.byref(out)))
    return out.value


def gs_model_pick(model: dict, candidates):
    n = len(candidates)
    c = (_i64 * n)(*[int(v) for v in candidates])
    best, tot = _i64(), ctypes.c_double()
    _check(_lib.gs_model_pick(ctypes.byref(_model_struct(model)), c, n, ctypes.byref(best), ctypes.byref(tot)))
    return best.value, tot.value


def gs_model_calibrate(ctx, n_iters: int, S_list, reps: int = 2) -> dict:
    n = len(S_list)
    c = (_i64 * n)(*[int(v) for v in S_list])
    out = gs_model()
    _check(_lib.gs_model_calibrate(ctx, n_iters, c, n, reps, ctypes.byref(out)), ctx)
    return _model_dict(out)


# ------------------------------------------------------- cost model --
GS_MLP_INPUTS, GS_MLP_HIDDEN, GS_MLP_PARAMS = 18, 32, 1697


class gs_workload(ctypes.Structure):
    _fields_ = [("kind", _i32), ("dtype", _i32), ("nx", _i64), ("ny", _i64), ("nz", _i64), ("n_iters", _i64)]


_sig("gs_features", [ctypes.POINTER(gs_workload), ctypes.POINTER(gs_tune_candidate), _i32, _fp])
_sig("gs_mlp_create", [ctypes.POINTER(_vp), ctypes.c_uint64, _vp])
_sig("gs_mlp_destroy", [_vp])
_sig("gs_mlp_last_error", [_vp], ctypes.c_char_p)
_sig("gs_mlp_set_params", [_vp, _fp, _i64])
_sig("gs_mlp_get_params", [_vp, _fp, _i64])
_sig("gs_mlp_fit_normalization", [_vp, _vp, _i64])
_sig("gs_mlp_set_normalization", [_vp, _fp, _fp])
_sig("gs_mlp_get_normalization", [_vp, _fp, _fp])
_sig("gs_mlp_loss_grad", [_vp, _vp, _vp, _i64, _fp, _fp])
_sig("gs_mlp_train", [_vp, _vp, _vp, _i64, _i32, _i32, ctypes.c_float, _fp])
_sig("gs_mlp_predict", [_vp, _vp, _i64, _vp])
_sig("gs_mlp_argmin", [_vp, _vp, _i64, ctypes.POINTER(_i64), _fp])
_sig("gs_mlp_argmin_ensemble", [ctypes.POINTER(_vp), ctypes.c_int32, _vp, _i64, ctypes.POINTER(_i64), _fp])


def _lcheck(st: int, m):
    if st != GS_OK:
        msg = _lib.gs_mlp_last_error(m).decode(errors="replace") if m else ""
        raise GsError(st, msg or _lib.gs_last_error(None).decode(errors="replace"))


def gs_features(workload: dict, candidates) -> np.ndarray:
    """Feature matrix (len(candidates) x GS_MLP_INPUTS, float32) of a workload dict
    (kind, dtype, nx, ny, nz, n_iters) with (plan dict, S) candidates."""
    w = gs_workload(*[int(workload[k]) for k, _ in gs_workload._fields_])
    n = len(candidates)
    arr = (gs_tune_candidate * n)()
    for i, (plan, S) in enumerate(candidates):
        arr[i].plan = gs_plan(*[int(plan.get(f, 0)) for f, _ in gs_plan._fields_])
        arr[i].batch_size = int(S)
    out = np.empty((n, GS_MLP_INPUTS), dtype=np.float32)
    _check(_lib.gs_features(ctypes.byref(w), arr, n, _f32_ptr(out)))
    return out


def gs_mlp_create(seed: int = 0, stream=None):
    h = _vp()
    _lcheck(_lib.gs_mlp_create(ctypes.byref(h), seed, _vp(stream) if stream else None), None)
    return h


def gs_mlp_destroy(m) -> None:
    _lcheck(_lib.gs_mlp_destroy(m), None)


def gs_mlp_last_error(m) -> str:
    return _lib.gs_mlp_last_error(m).decode(errors="replace")


def gs_mlp_set_params(m, params: np.ndarray) -> None:
    _lcheck(_lib.gs_mlp_set_params(m, _f32_ptr(params), params.size), m)


def gs_mlp_get_params(m) -> np.ndarray:
    out = np.empty(GS_MLP_PARAMS, dtype=np.float32)
    _lcheck(_lib.gs_mlp_get_params(m, _f32_ptr(out), out.size), m)
    return out


def gs_mlp_fit_normalization(m, X_dev_ptr: int, n_rows: int) -> None:
    _lcheck(_lib.gs_mlp_fit_normalization(m, _vp(X_dev_ptr), n_rows), m)


def gs_mlp_set_normalization(m, mean: np.ndarray, inv_std: np.ndarray) -> None:
    _lcheck(_lib.gs_mlp_set_normalization(m, _f32_ptr(mean), _f32_ptr(inv_std)), m)


def gs_mlp_get_normalization(m):
    mean = np.empty(GS_MLP_INPUTS, dtype=np.float32)
    inv = np.empty(GS_MLP_INPUTS, dtype=np.float32)
    _lcheck(_lib.gs_mlp_get_normalization(m, _f32_ptr(mean), _f32_ptr(inv)), m)
    return mean, inv


def gs_mlp_loss_grad(m, X_dev_ptr: int, y_dev_ptr: int, n_rows: int):
    loss = ctypes.c_float()
    grad = np.empty(GS_MLP_PARAMS, dtype=np.float32)
    _lcheck(_lib.gs_mlp_loss_grad(m, _vp(X_dev_ptr), _vp(y_dev_ptr), n_rows, ctypes.byref(loss), _f32_ptr(grad)), m)
    return loss.value, grad


def gs_mlp_train(m, X_dev_ptr: int, y_dev_ptr: int, n_rows: int, epochs: int, batch_rows: int, lr: float) -> float:
    loss = ctypes.c_float()
    _lcheck(_lib.gs_mlp_train(m, _vp(X_dev_ptr), _vp(y_dev_ptr), n_rows, epochs, batch_rows, lr, ctypes.byref(loss)),
            m)
    return loss.value


def gs_mlp_predict(m, X_dev_ptr: int, n_rows: int, pred_dev_ptr: int) -> None:
    _lcheck(_lib.gs_mlp_predict(m, _vp(X_dev_ptr), n_rows, _vp(pred_dev_ptr)), m)


def gs_mlp_argmin(m, X_dev_ptr: int, n_rows: int):
    idx = _i64()
    val = ctypes.c_float()
    _lcheck(_lib.gs_mlp_argmin(m, _vp(X_dev_ptr), n_rows, ctypes.byref(idx), ctypes.byref(val)), m)
    return idx.value, val.value


def gs_mlp_argmin_ensemble(models, X_dev_ptr: int, n_rows: int):
    """Row with the smallest mean prediction of several models, and that mean."""
    arr = (_vp * len(models))(*models)
    idx = _i64()
    val = ctypes.c_float()
    _lcheck(_lib.gs_mlp_argmin_ensemble(arr, len(models), _vp(X_dev_ptr), n_rows, ctypes.byref(idx),
                                        ctypes.byref(val)), models[0] if models else None)
    return idx.value, val.value


# ------------------------------------- choosing the plan and batch size --
_sig("gs_plan_check", [ctypes.POINTER(gs_workload), ctypes.POINTER(gs_plan), ctypes.POINTER(gs_plan)])
_sig("gs_candidates", [ctypes.POINTER(gs_workload), ctypes.POINTER(gs_tune_candidate), _i32, ctypes.POINTER(_i32)])
_sig("gs_pick", [ctypes.POINTER(_vp), _i32, ctypes.POINTER(gs_workload), ctypes.POINTER(gs_tune_candidate), _fp])
_sig("gs_pick_analytic", [_vp, _i64, _i32, ctypes.POINTER(_i64), ctypes.POINTER(gs_model)])

_SHAPE = ("block_x", "rows", "temporal_depth", "kernel", "tile_y")  # the plan fields a candidate sets


def _workload(workload: dict):
    return gs_workload(*[int(workload.get(k, 1) if k == "n_iters" else workload[k]) for k, _ in gs_workload._fields_])


def gs_plan_check(workload: dict, plan: dict) -> dict:
    """The plan as gs_set_plan would apply it on a context of the workload
    (kind, dtype, nx, ny, nz), defaults filled in; GsError if refused."""
    p = gs_plan(*[int(plan.get(f, 0)) for f, _ in gs_plan._fields_])
    out = gs_plan()
    _check(_lib.gs_plan_check(ctypes.byref(_workload(workload)), ctypes.byref(p), ctypes.byref(out)))
    return {n: getattr(out, n) for n, _ in gs_plan._fields_}


def gs_candidates(workload: dict):
    """The (plan dict of block_x, rows, temporal_depth, kernel, tile_y; S)
    pairs the pickers choose from, plan after plan."""
    w = _workload(workload)
    n = _i32()
    _check(_lib.gs_candidates(ctypes.byref(w), None, 0, ctypes.byref(n)))
    arr = (gs_tune_candidate * n.value)()
    _check(_lib.gs_candidates(ctypes.byref(w), arr, n.value, ctypes.byref(n)))
    return [({f: getattr(c.plan, f) for f in _SHAPE}, c.batch_size) for c in arr]


def gs_pick(models, workload: dict):
    """The learned choice for a run of workload["n_iters"] iterations:
    (plan dict, S, predicted ms per iteration)."""
    arr = (_vp * len(models))(*models)
    best = gs_tune_candidate()
    pred = ctypes.c_float()
    _lcheck(_lib.gs_pick(arr, len(models), ctypes.byref(_workload(workload)), ctypes.byref(best),
                         ctypes.byref(pred)), models[0] if models else None)
    return {f: getattr(best.plan, f) for f in _SHAPE}, best.batch_size, pred.value


_sig("gs_mlp_create_builtin", [ctypes.POINTER(_vp), _i32, _vp])
_sig("gs_mlp_builtin_info", [], ctypes.c_char_p)
_sig("gs_pick_ctx", [_vp, _i64, ctypes.POINTER(gs_plan), ctypes.POINTER(_i64), _fp])
GS_MLP_BUILTIN_MEMBERS = 3


def gs_mlp_create_builtin(member: int, stream=None):
    """Member `member` of the trained ensemble compiled into the library."""
    h = _vp()
    st = _lib.gs_mlp_create_builtin(ctypes.byref(h), member, _vp(stream) if stream else None)
    if st != GS_OK:
        raise GsError(st, _lib.gs_last_error(None).decode(errors="replace"))
    return h


def gs_mlp_builtin_info() -> str:
    return _lib.gs_mlp_builtin_info().decode(errors="replace")


def gs_pick_ctx(ctx, n_iters: int):
    """The learned choice for a run of n_iters iterations of ctx's workload
    with the library's own ensemble, applied to ctx: (plan dict as applied,
    S, predicted ms per iteration)."""
    p = gs_plan()
    S = _i64()
    pred = ctypes.c_float()
    _check(_lib.gs_pick_ctx(ctx, int(n_iters), ctypes.byref(p), ctypes.byref(S), ctypes.byref(pred)), ctx)
    return {n: getattr(p, n) for n, _ in gs_plan._fields_}, S.value, pred.value


def gs_pick_analytic(ctx, n_iters: int, reps: int = 2):
    """The paper's choice on a context at its current plan: (S, fitted model)."""
    S = _i64()
    m = gs_model()
    _check(_lib.gs_pick_analytic(ctx, int(n_iters), int(reps), ctypes.byref(S), ctypes.byref(m)), ctx)
    return S.value, _model_dict(m)


# ----------------------------------------------------- instance batches --
GS_MULTI_FUSED, GS_MULTI_SEPARATE = range(2)


def _mcheck(st: int, m):
    if st != GS_OK:
        raise GsError(st, _lib.gs_multi_last_error(m).decode(errors="replace") if m else "")


def gs_multi_create(nx, ny, dtype: int = GS_F32, bc: int = GS_BC_CLAMP, stream=None):
    n = len(nx)
    ax = (_i64 * n)(*[int(v) for v in nx])
    ay = (_i64 * n)(*[int(v) for v in ny])
    h = _vp()
    st = _lib.gs_multi_create(ctypes.byref(h), n, ax, ay, dtype, bc, _vp(stream) if stream else None)
    if st != GS_OK:
        raise GsError(st, "gs_multi_create failed: " + _lib.gs_last_error(None).decode(errors="replace"))
    return h


def gs_multi_destroy(m) -> None:
    _mcheck(_lib.gs_multi_destroy(m), None)


def gs_multi_last_error(m) -> str:
    return _lib.gs_multi_last_error(m).decode(errors="replace")


def gs_multi_set_heat_coeffs(m, k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.05, t_amb=80.0) -> None:
    c = gs_heat_coeffs(k, cx, cy, cz, cz2, t_amb)
    _mcheck(_lib.gs_multi_set_heat_coeffs(m, ctypes.byref(c)), m)


def gs_multi_set_plan(m, block_x=0, rows=0, blocks=0, use_pdl=0, kernel=0, traverse=0, temporal_depth=0) -> None:
    p = gs_multi_plan(block_x, rows, blocks, use_pdl, kernel, traverse, temporal_depth)
    _mcheck(_lib.gs_multi_set_plan(m, ctypes.byref(p)), m)


def gs_multi_bind_field(m, i: int, field: int, ptr: int, pitch: int) -> None:
    _mcheck(_lib.gs_multi_bind_field(m, i, field, _vp(ptr) if ptr else None, pitch), m)


def gs_multi_upload(m, i: int, field: int, host: np.ndarray) -> None:
    _mcheck(_lib.gs_multi_upload(m, i, field, _f32_ptr(host), host.size), m)


def gs_multi_read_field(m, i: int, field: int, out: np.ndarray) -> np.ndarray:
    _mcheck(_lib.gs_multi_read_field(m, i, field, _f32_ptr(out), out.size), m)
    return out


def gs_multi_step(m, n_iters: int, batch_size: int, mode: int = GS_MULTI_FUSED) -> None:
    _mcheck(_lib.gs_multi_step(m, n_iters, batch_size, mode), m)


def gs_multi_get_parity(m) -> int:
    v = _i32()
    _mcheck(_lib.gs_multi_get_parity(m, ctypes.byref(v)), m)
    return v.value


def gs_multi_sync(m) -> None:
    _mcheck(_lib.gs_multi_sync(m), m)


def gs_multi_get_stats(m) -> dict:
    s = gs_stats()
    _mcheck(_lib.gs_multi_get_stats(m, ctypes.byref(s)), m)
    return {n: getattr(s, n) for n, _ in gs_stats._fields_}


# --------------------------------------------------- slab decomposition --
_sig("gs_slab_create", [ctypes.POINTER(_vp), ctypes.c_int, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int, _i32, _i32,
                        _vp])
_sig("gs_slab_destroy", [_vp])
_sig("gs_slab_last_error", [_vp], ctypes.c_char_p)
_sig("gs_slab_extent", [_vp, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)])
_sig("gs_slab_set_heat_coeffs", [_vp, ctypes.POINTER(gs_heat_coeffs)])
_sig("gs_slab_set_fdtd_params", [_vp, ctypes.POINTER(gs_fdtd_params)])
_sig("gs_slab_set_plan", [_vp, ctypes.POINTER(gs_plan)])
_sig("gs_slab_upload", [_vp, ctypes.c_int, _fp, _i64])
_sig("gs_slab_read_field", [_vp, ctypes.c_int, _fp, _i64])
_sig("gs_slab_step", [_vp, _i64, _i64])
_sig("gs_slab_set_time", [_vp, _i64])
_sig("gs_slab_sync", [_vp])
_sig("gs_slab_get_stats", [_vp, ctypes.POINTER(gs_stats)])


def _scheck(st: int, s):
    if st != GS_OK:
        msg = _lib.gs_slab_last_error(s).decode(errors="replace") if s else ""
        raise GsError(st, msg or _lib.gs_last_error(None).decode(errors="replace"))


def gs_slab_create(kind: int, nx: int, ny: int, nz: int, n_slabs: int, halo: int = 1, dtype: int = GS_F32,
                   bc: int = GS_BC_CLAMP, stream=None):
    h = _vp()
    st = _lib.gs_slab_create(ctypes.byref(h), kind, nx, ny, nz, dtype, bc, n_slabs, halo,
                             _vp(stream) if stream else None)
    if st != GS_OK:
        raise GsError(st, _lib.gs_last_error(None).decode(errors="replace"))
    return h


def gs_slab_destroy(s) -> None:
    _scheck(_lib.gs_slab_destroy(s), None)


def gs_slab_last_error(s) -> str:
    return _lib.gs_slab_last_error(s).decode(errors="replace")


def gs_slab_extent(s, k: int):
    """(first, count) of the rows/planes slab k owns."""
    a, b = _i64(), _i64()
    _scheck(_lib.gs_slab_extent(s, k, ctypes.byref(a), ctypes.byref(b)), None)
    return a.value, b.value


def gs_slab_set_heat_coeffs(s, k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.05, t_amb=80.0) -> None:
    c = gs_heat_coeffs(k, cx, cy, cz, cz2, t_amb)
    _scheck(_lib.gs_slab_set_heat_coeffs(s, ctypes.byref(c)), s)


def gs_slab_set_fdtd_params(s, courant=0.5, src_on=0, src=(0, 0, 0), amp=1.0, delay=60.0, width=20.0) -> None:
    p = gs_fdtd_params(courant, src_on, src[0], src[1], src[2], amp, delay, width)
    _scheck(_lib.gs_slab_set_fdtd_params(s, ctypes.byref(p)), s)


def gs_slab_set_plan(s, block_x=0, rows=0, tile_x=0, tile_y=0, temporal_depth=0, use_pdl=0, device_launch=0,
                     kernel=0, graph_loop=0, traverse=0) -> None:
    p = gs_plan(block_x, rows, tile_x, tile_y, temporal_depth, use_pdl, device_launch, kernel, graph_loop, traverse)
    _scheck(_lib.gs_slab_set_plan(s, ctypes.byref(p)), s)


def gs_slab_upload(s, field: int, host: np.ndarray) -> None:
    _scheck(_lib.gs_slab_upload(s, field, _f32_ptr(host), host.size), s)


def gs_slab_read_field(s, field: int, out: np.ndarray) -> np.ndarray:
    _scheck(_lib.gs_slab_read_field(s, field, _f32_ptr(out), out.size), s)
    return out


def gs_slab_step(s, n_iters: int, batch_size: int) -> None:
    _scheck(_lib.gs_slab_step(s, n_iters, batch_size), s)


def gs_slab_set_time(s, n: int) -> None:
    _scheck(_lib.gs_slab_set_time(s, n), s)


def gs_slab_sync(s) -> None:
    _scheck(_lib.gs_slab_sync(s), s)


def gs_slab_get_stats(s) -> dict:
    st = gs_stats()
    _scheck(_lib.gs_slab_get_stats(s, ctypes.byref(st)), s)
    return {n: getattr(st, n) for n, _ in gs_stats._fields_}


class gs_multi_tune_candidate(ctypes.Structure):
    _fields_ = [("plan", gs_multi_plan), ("batch_size", ctypes.c_int64)]


class gs_multi_tune_result(ctypes.Structure):
    _fields_ = [("plan", gs_multi_plan), ("batch_size", ctypes.c_int64), ("build_seconds", ctypes.c_double),
                ("exec_ms_per_iter", ctypes.c_double), ("total_ms", ctypes.c_double), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_sig("gs_multi_candidates", [_vp, ctypes.POINTER(gs_multi_tune_candidate), _i32, ctypes.POINTER(_i32)])
_sig("gs_multi_autotune", [_vp, _i64, _i32, ctypes.POINTER(gs_multi_tune_candidate), _i32,
                           ctypes.POINTER(gs_multi_tune_result), ctypes.POINTER(_i32)])
_sig("gs_multi_get_plan", [_vp, ctypes.POINTER(gs_multi_plan)])


def _mplan_dict(p) -> dict:
    return {n: getattr(p, n) for n, _ in gs_multi_plan._fields_}


def gs_multi_get_plan(m) -> dict:
    p = gs_multi_plan()
    _mcheck(_lib.gs_multi_get_plan(m, ctypes.byref(p)), m)
    return _mplan_dict(p)


def gs_multi_candidates(m):
    """The (plan dict, S) pairs the batch's tuner sweeps."""
    n = _i32()
    _mcheck(_lib.gs_multi_candidates(m, None, 0, ctypes.byref(n)), m)
    arr = (gs_multi_tune_candidate * n.value)()
    _mcheck(_lib.gs_multi_candidates(m, arr, n.value, ctypes.byref(n)), m)
    return [(_mplan_dict(c.plan), c.batch_size) for c in arr]


def gs_multi_autotune(m, n_iters: int, candidates, reps: int = 3):
    """candidates: list of (plan dict, batch_size).  Returns (results, best
    index); each result a dict with the plan as applied, batch_size,
    build_seconds, exec_ms_per_iter, total_ms and status."""
    n = len(candidates)
    arr = (gs_multi_tune_candidate * n)()
    for i, (plan, S) in enumerate(candidates):
        arr[i].plan = gs_multi_plan(*[int(plan.get(f, 0)) for f, _ in gs_multi_plan._fields_])
        arr[i].batch_size = int(S)
    res = (gs_multi_tune_result * n)()
    best = _i32(-1)
    _mcheck(_lib.gs_multi_autotune(m, n_iters, reps, arr, n, res, ctypes.byref(best)), m)
    out = [dict(plan=_mplan_dict(r.plan), batch_size=r.batch_size, build_seconds=r.build_seconds,
                exec_ms_per_iter=r.exec_ms_per_iter, total_ms=r.total_ms, status=r.status) for r in res]
    return out, best.value


# ------------------------------------------------- step without allocation --
GS_NOALLOC_MAX_INSTANCES = 256


class gs_instance(ctypes.Structure):
    _fields_ = [("T0", _vp), ("T1", _vp), ("P", _vp), ("nx", _i64), ("ny", _i64), ("pitch", _i64),
                ("p_pitch", _i64)]


_sig("gs_multi_step_noalloc", [ctypes.POINTER(gs_instance), _i32, _i32, _i64, ctypes.POINTER(gs_heat_coeffs),
                               ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_i32)])


def gs_multi_step_noalloc(instances, parity: int, n_iters: int, coeffs=None, dtype: int = GS_F32,
                          bc: int = GS_BC_CLAMP, stream=None) -> int:
    """instances: list of dicts with T0, T1, P (device pointers), nx, ny,
    pitch, p_pitch.  Returns the parity after the call."""
    n = len(instances)
    arr = (gs_instance * max(n, 1))()
    for i, d in enumerate(instances):
        arr[i] = gs_instance(d["T0"], d["T1"], d["P"], d["nx"], d["ny"], d["pitch"], d["p_pitch"])
    c = gs_heat_coeffs(**(coeffs or dict(k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.05, t_amb=80.0)))
    out = _i32(parity)
    _check(_lib.gs_multi_step_noalloc(arr, n, parity, n_iters, ctypes.byref(c), dtype, bc,
                                      _vp(stream) if stream else None, ctypes.byref(out)))
    return out.value


# ------------------------------------------------------- fault injection --
GS_INJECT_NONE, GS_INJECT_MALLOC, GS_INJECT_GRAPH_NODE = range(3)
_sig("gs_debug_inject_failure", [ctypes.c_int, _i64])
_sig("gs_debug_injection_pending", [ctypes.POINTER(_i32)])


def gs_debug_inject_failure(call: int, after: int = 0) -> None:
    """Make the library's (after+1)-th next call of kind `call` fail once."""
    _check(_lib.gs_debug_inject_failure(call, after))


_sig("gs_debug_checked_build", [], ctypes.c_int)
_sig("gs_debug_check_ranges", [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _i32])
_sig("gs_debug_check_read", [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)])
_sig("gs_debug_owned_ranges", [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _i32,
                               ctypes.POINTER(_i32)])
GS_CHECK_MAX_RANGES = 128


def gs_debug_owned_ranges(ctx):
    """(lo, hi) byte ranges of the device memory ctx owns that its kernels touch."""
    lo = (ctypes.c_uint64 * 8)()
    hi = (ctypes.c_uint64 * 8)()
    n = _i32()
    _check(_lib.gs_debug_owned_ranges(ctx, lo, hi, 8, ctypes.byref(n)), ctx)
    return [(lo[i], hi[i]) for i in range(min(n.value, 8))]


def gs_debug_checked_build() -> bool:
    return bool(_lib.gs_debug_checked_build())


def gs_debug_check_ranges(ranges) -> None:
    """ranges: (lo, hi) byte addresses of device memory the kernels may touch."""
    n = len(ranges)
    lo = (ctypes.c_uint64 * max(n, 1))(*[int(r[0]) for r in ranges])
    hi = (ctypes.c_uint64 * max(n, 1))(*[int(r[1]) for r in ranges])
    _check(_lib.gs_debug_check_ranges(lo, hi, n))


def gs_debug_check_read():
    """(refused accesses since the last read, first refused address)."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.gs_debug_check_read(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


_sig("gs_wait_timeouts", [ctypes.POINTER(ctypes.c_uint64)])


def gs_wait_timeouts() -> int:
    """Blocks of the library's kernels whose bounded wait ran out since the
    last call (the count is cleared; synchronises the device)."""
    n = ctypes.c_uint64()
    _check(_lib.gs_wait_timeouts(ctypes.byref(n)))
    return n.value


def gs_debug_injection_pending() -> bool:
    v = _i32()
    _check(_lib.gs_debug_injection_pending(ctypes.byref(v)))
    return bool(v.value)


def raw_call(name: str, *args) -> int:
    """Call a C entry point by name with ctypes arguments; returns its status
    (no exception).  Used by tests that check error returns."""
    return int(getattr(_lib, name)(*args))


from .fields import FdtdFields, HeatFields, MultiFields  # noqa: E402  (device-memory helpers)

__all__ = [n for n in dir() if n.startswith(("gs_", "GS_"))] + ["GsError", "HeatFields", "FdtdFields", "MultiFields"]
