"""FP64 CPU oracle for the stencil time stepping (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's product path never loads
it, and it shares no code with the CUDA path.

What it computes (all in float64, plain loops in ``oracle.c``):

* ``heat_run``: n explicit thermal steps, 2D 5-point or 3D 7-point.  The
  paper runs Rodinia Hotspot and Hotspot3D (Sec. III-C, Fig. 7) without
  printing their update; the update used here is
  ``T' = T + k*(P + cy*(N+S-2T) + cx*(E+W-2T) + cz*(t_amb-T) [+ cz2*(U+D-2T)])``
  with clamp (zero-flux) or Dirichlet-0 boundaries, P acting on layer 0 only
  in 3D.
* ``fdtd_run``: n Yee leapfrog steps (H update, then E update, then a soft
  Ez point source), the paper's FDTD Maxwell solver with its two kernels per
  step (Sec. III-C), PEC cavity, normalised units; optionally in linear,
  lossy media given by a per-cell material map (the textbook lossy-medium
  Yee update).
* Batching iterations into graphs (Sec. III-A, Listings 1-3) does not change
  the result, so no oracle function models graphs: the oracle of a batched run
  is the plain run.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms (heat eigenmode decay, uniform relaxation, Yee energy
invariance, Yee cavity dispersion, the cavity-mode recurrence in a uniform
lossy medium), invariants (the permittivity-weighted Yee energy in a
lossless heterogeneous medium) and a brute-force matrix restatement.  The
source-driven FDTD field has no closed form; it is pinned through the source
value, the mirror/swap symmetries, the same scheme's source-free pins and,
step by step, the discrete energy budget of the soft source
(W^{n+1} - W^n = g(n) (Ez^{n+1} + Ez^n) at the source; in a lossy medium
with the Joule terms and the source cell's (eps + s sigma / 2) factor); its
5000-step field values themselves stay parity unpinned.
``tests/test_oracle_mutations.py`` plants plausible mistakes in a copy of
``oracle.c`` (selected with the GS_ORACLE_SRC environment variable) and
checks that a pin fails for each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GS_ORACLE_SRC names another copy of oracle.c, built beside it: the oracle's
# mutation test plants a mistake in such a copy and checks that a pin fails.
_SRC = os.environ.get("GS_ORACLE_SRC") or os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(_SRC)), "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_CLAMP = 0
BC_DIRICHLET0 = 1

# Coefficients of the thermal workloads (2D: cz2 unused).
HEAT_COEFFS_2D = dict(k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.0, t_amb=80.0)
HEAT_COEFFS_3D = dict(k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.05, t_amb=80.0)


class _HeatCoeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("k", "cx", "cy", "cz", "cz2", "t_amb")]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    # GS_ORACLE_CFLAGS: extra compiler flags (the sanitizer test builds a copy
    # with -fsanitize=address,undefined)
    extra = os.environ.get("GS_ORACLE_CFLAGS", "").split()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra, _SRC, "-o", _LIB_PATH + ".tmp",
            "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.or_heat_run.argtypes = [i64, i64, i64, i64, dp, dp, ctypes.POINTER(_HeatCoeffs), ctypes.c_int]
            lib.or_heat_run.restype = ctypes.c_int
            lib.or_fdtd_run.argtypes = [i64, i64, i64, ctypes.c_double] + [dp] * 6 + [
                ctypes.c_int, i64, i64, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.or_fdtd_run.restype = None
            lib.or_fdtd_run_media.argtypes = [i64, i64, i64, ctypes.c_double] + [dp] * 6 + [
                ctypes.POINTER(ctypes.c_uint8), ctypes.c_int, dp, dp, dp, dp,
                ctypes.c_int, i64, i64, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.or_fdtd_run_media.restype = ctypes.c_int
            lib.or_fdtd_source.argtypes = [ctypes.c_double] * 4
            lib.or_fdtd_source.restype = ctypes.c_double
            lib.or_num_threads.argtypes = []
            lib.or_num_threads.restype = ctypes.c_int
            lib.or_set_num_threads.argtypes = [ctypes.c_int]
            lib.or_set_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    """Threads the oracle's loops run on (OpenMP; 1 without it)."""
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> int:
    """Threads of the oracle's later loops in the calling thread; returns the
    count now in effect."""
    return int(_load().or_set_num_threads(int(n)))


def heat_run(T0, P, n_steps: int, coeffs: dict, bc: int = BC_CLAMP) -> np.ndarray:
    """Return the thermal field after ``n_steps`` explicit steps.

    ``T0``: (ny, nx) for the 2D 5-point stencil or (nz, ny, nx) for the 3D
    7-point stencil.  ``P``: (ny, nx) power map (layer 0 only in 3D).  Inputs
    are promoted to float64; the returned array is float64.
    """
    T = np.array(T0, dtype=np.float64, order="C", copy=True)
    Pd = np.ascontiguousarray(P, dtype=np.float64)
    if T.ndim == 2:
        nz, (ny, nx) = 1, T.shape
    elif T.ndim == 3:
        nz, ny, nx = T.shape
    else:
        raise ValueError("T0 must be 2D or 3D")
    if Pd.shape != (ny, nx):
        raise ValueError(f"P must have shape {(ny, nx)}, got {Pd.shape}")
    c = _HeatCoeffs(*(float(coeffs[n]) for n in ("k", "cx", "cy", "cz", "cz2", "t_amb")))
    if T.size == 0 or n_steps == 0:
        return T
    rc = _load().or_heat_run(nx, ny, nz, int(n_steps), _dptr(T), _dptr(Pd), ctypes.byref(c), int(bc))
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return T


FDTD_COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def fdtd_zero_fields(N: int) -> dict:
    """Six zero (N+1)^3 float64 arrays indexed [k][j][i]."""
    return {c: np.zeros((N + 1, N + 1, N + 1), dtype=np.float64) for c in FDTD_COMPONENTS}


def fdtd_source(n, amp=1.0, delay=60.0, width=20.0) -> float:
    """Soft-source amplitude amp*exp(-((n-delay)/width)^2) at step n."""
    return float(_load().or_fdtd_source(float(n), float(amp), float(delay), float(width)))


def fdtd_run(fields: dict, N: int, n_steps: int, courant: float = 0.5, n0: int = 0,
             src=None, amp=1.0, delay=60.0, width=20.0, media=None) -> dict:
    """Advance the six Yee components in place by ``n_steps`` leapfrog steps.

    ``fields``: dict of six float64 (N+1)^3 arrays (see ``FDTD_COMPONENTS``),
    H holding H^{n0-1/2} and E holding E^{n0}.  ``src``: (i, j, k) of the soft
    Ez source, or None for a source-free run.  ``media``: None (vacuum) or
    ``(mat, table)`` with ``mat`` a uint8 (N+1)^3 material-id array indexed
    [k][j][i] and ``table`` a sequence of (eps_r, sigma, mu_r, sigma_m) rows
    (at most 256; ids past the table are vacuum).  Returns ``fields``.
    """
    arrs = []
    for c in FDTD_COMPONENTS:
        a = fields[c]
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.shape != (N + 1,) * 3:
            raise ValueError(f"{c}: need a C-contiguous float64 array of shape {(N + 1,) * 3}")
        arrs.append(a)
    si, sj, sk = src if src is not None else (0, 0, 0)
    if media is None:
        _load().or_fdtd_run(N, int(n0), int(n_steps), float(courant), *[_dptr(a) for a in arrs],
                            1 if src is not None else 0, si, sj, sk, float(amp), float(delay), float(width))
        return fields
    mat, table = media
    mat = np.ascontiguousarray(mat, dtype=np.uint8)
    if mat.shape != (N + 1,) * 3:
        raise ValueError(f"material map: need shape {(N + 1,) * 3}")
    tab = np.array(table, dtype=np.float64).reshape(-1, 4)
    if len(tab) > 256:
        raise ValueError("at most 256 materials")
    cols = [np.ascontiguousarray(tab[:, q]) for q in range(4)]
    rc = _load().or_fdtd_run_media(N, int(n0), int(n_steps), float(courant), *[_dptr(a) for a in arrs],
                                   mat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(tab),
                                   *[_dptr(c) for c in cols], 1 if src is not None else 0, si, sj, sk,
                                   float(amp), float(delay), float(width))
    if rc != 0:
        raise ValueError("bad material table")
    return fields


def skeleton_run(x0, c: float, n_steps: int) -> np.ndarray:
    """The paper's skeleton application (Sec. III-C): the vector multiplied
    by the constant c once per iteration, n_steps times, in float64."""
    x = np.array(x0, dtype=np.float64, copy=True)
    for _ in range(int(n_steps)):
        x = c * x
    return x
