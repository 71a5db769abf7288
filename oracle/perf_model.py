"""Oracle of the paper's performance model (Sec. III-B, Eqs. 1-6).

TEST INFRASTRUCTURE ONLY: the tests use it to check the library's
gs_model_* entry points; the library never imports it.

* Eq. 1: T = T_C + T_E.
* Eq. 2: T_C = k_c S + b_c (graph creation grows linearly with the nodes).
* Eq. 3: T_E = T_l + (T_k S + T_i (S - 1)) I + T_a (I - 1), with
  Eq. 4: I = I_k / S graph launches.
* Eq. 5/6: substituting Eq. 4 into Eq. 3 gives T_E = a/S + b with
  a = I_k (T_a - T_i) and b = I_k (T_k + T_i) - T_a + T_l.
* The batch size is chosen to minimise Eq. 1 over the admissible integer S
  (Sec. III-B: S must divide I_k).
Fits are ordinary least squares (numpy.linalg.lstsq) on the design matrices
[S, 1] (Eq. 2) and [1/S, 1] (Eq. 6).
"""
from __future__ import annotations

import numpy as np


def creation_time(k_c, b_c, S):
    """Eq. 2."""
    return k_c * np.asarray(S, dtype=np.float64) + b_c


def exec_time_eq3(T_l, T_k, T_i, T_a, S, I_k):
    """Eq. 3 with Eq. 4 (I = I_k / S)."""
    S = np.asarray(S, dtype=np.float64)
    I = I_k / S
    return T_l + (T_k * S + T_i * (S - 1.0)) * I + T_a * (I - 1.0)


def exec_coeffs(T_l, T_k, T_i, T_a, I_k):
    """Eq. 6's a and b from the timing constants (Eq. 5)."""
    return I_k * (T_a - T_i), I_k * (T_k + T_i) - T_a + T_l


def exec_time_eq6(a, b, S):
    """Eq. 6."""
    return a / np.asarray(S, dtype=np.float64) + b


def total_time(model, S):
    """Eq. 1 with Eqs. 2 and 6."""
    return creation_time(model["k_c"], model["b_c"], S) + exec_time_eq6(model["a"], model["b"], S)


def fit(S, t_create, t_exec):
    """Least-squares fits of Eq. 2 and Eq. 6; returns k_c, b_c, a, b and the
    mean absolute errors of both fits."""
    S = np.asarray(S, dtype=np.float64)
    tc = np.asarray(t_create, dtype=np.float64)
    te = np.asarray(t_exec, dtype=np.float64)
    (k_c, b_c), *_ = np.linalg.lstsq(np.stack([S, np.ones_like(S)], 1), tc, rcond=None)
    (a, b), *_ = np.linalg.lstsq(np.stack([1.0 / S, np.ones_like(S)], 1), te, rcond=None)
    return dict(k_c=float(k_c), b_c=float(b_c), a=float(a), b=float(b),
                mae_create=float(np.mean(np.abs(k_c * S + b_c - tc))),
                mae_exec=float(np.mean(np.abs(a / S + b - te))))


def pick(model, candidates):
    """The candidate batch size with the smallest Eq. 1 total (ties: smaller S)."""
    cands = sorted(int(c) for c in candidates)
    totals = [float(total_time(model, c)) for c in cands]
    i = int(np.argmin(totals))  # first minimum = smallest S among ties
    return cands[i], totals[i]


def divisors(I_k):
    """Batch sizes the paper admits for I_k kernel executions (S | I_k)."""
    return [d for d in range(1, I_k + 1) if I_k % d == 0]
