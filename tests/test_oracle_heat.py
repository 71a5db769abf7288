"""Pins for the FP64 thermal oracle (CPU only).

The oracle is checked against things that do not come from itself:
closed-form eigenmode decay (Dirichlet sine modes, clamp cosine modes),
uniform relaxation toward t_amb + P/cz, conservation of the total heat, the
discrete maximum principle, and a brute-force matrix restatement of the
update on tiny grids.  Coefficients differ per axis (cx != cy != cz2) and the
grids are not square, so a swapped axis, a dropped term or a wrong sign fails
at least one pin.
"""
import math

import numpy as np
import pytest

import gs_inputs

pytestmark = []

ASYM = dict(k=0.5, cx=0.1, cy=0.13, cz=0.0, cz2=0.07, t_amb=80.0)


def _sin2(m, n):
    return math.sin(math.pi * m / (2.0 * n)) ** 2


def test_dirichlet_sine_eigenmode_2d(oracle):
    # Source-free, cz = 0, zero ghosts: the sine mode (kx, ky) decays by
    # [1 - 4k(cx sin^2(pi kx/2(nx+1)) + cy sin^2(pi ky/2(ny+1)))]^n exactly.
    nx, ny, n = 31, 23, 1000
    for kx, ky in ((1, 1), (2, 1), (1, 3)):
        x = np.arange(nx)
        y = np.arange(ny)
        T0 = np.outer(np.sin(math.pi * ky * (y + 1) / (ny + 1)), np.sin(math.pi * kx * (x + 1) / (nx + 1)))
        P = np.zeros((ny, nx))
        lam = 1.0 - 4.0 * ASYM["k"] * (ASYM["cx"] * _sin2(kx, nx + 1) + ASYM["cy"] * _sin2(ky, ny + 1))
        Tn = oracle.heat_run(T0, P, n, ASYM, oracle.BC_DIRICHLET0)
        expect = lam ** n * T0
        assert np.max(np.abs(Tn - expect)) <= 1e-12 * lam ** n * np.max(np.abs(T0))


def test_dirichlet_sine_eigenmode_3d(oracle):
    nx, ny, nz, n = 13, 11, 7, 300
    kx, ky, kz = 1, 2, 1
    sx = np.sin(math.pi * kx * (np.arange(nx) + 1) / (nx + 1))
    sy = np.sin(math.pi * ky * (np.arange(ny) + 1) / (ny + 1))
    sz = np.sin(math.pi * kz * (np.arange(nz) + 1) / (nz + 1))
    T0 = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    P = np.zeros((ny, nx))
    c = ASYM
    lam = 1.0 - 4.0 * c["k"] * (c["cx"] * _sin2(kx, nx + 1) + c["cy"] * _sin2(ky, ny + 1)
                                + c["cz2"] * _sin2(kz, nz + 1))
    Tn = oracle.heat_run(T0, P, n, c, oracle.BC_DIRICHLET0)
    assert np.max(np.abs(Tn - lam ** n * T0)) <= 1e-12 * lam ** n


# Rounding floor of a field that sits near t_amb = 80: one ulp(80) per step,
# remembered for about 1/(k cz) = 200 steps by the (1 - k cz) decay.
_AMB_FLOOR = 200 * np.spacing(80.0)


def test_clamp_cosine_mode_with_ambient_2d(oracle):
    # Clamp = zero flux: cos(pi kx (x+1/2)/nx) modes; the ambient term adds
    # the factor (1 - k cz) around t_amb.
    nx, ny, n = 24, 17, 1000
    c = dict(oracle.HEAT_COEFFS_2D, cy=0.13)
    for kx, ky in ((1, 0), (0, 1), (2, 3)):
        cx_ = np.cos(math.pi * kx * (np.arange(nx) + 0.5) / nx)
        cy_ = np.cos(math.pi * ky * (np.arange(ny) + 0.5) / ny)
        mode = np.outer(cy_, cx_)
        T0 = 80.0 + 5.0 * mode
        mu = 1.0 - c["k"] * c["cz"] - 4.0 * c["k"] * (c["cx"] * _sin2(kx, nx) + c["cy"] * _sin2(ky, ny))
        Tn = oracle.heat_run(T0, np.zeros((ny, nx)), n, c, oracle.BC_CLAMP)
        assert np.max(np.abs((Tn - 80.0) - mu ** n * 5.0 * mode)) <= 1e-11 * mu ** n * 5.0 + _AMB_FLOOR


def test_clamp_cosine_mode_3d(oracle):
    nx, ny, nz, n = 12, 10, 6, 200
    c = dict(oracle.HEAT_COEFFS_3D, cy=0.13)
    kx, ky, kz = 1, 2, 1
    mode = (np.cos(math.pi * kz * (np.arange(nz) + 0.5) / nz)[:, None, None]
            * np.cos(math.pi * ky * (np.arange(ny) + 0.5) / ny)[None, :, None]
            * np.cos(math.pi * kx * (np.arange(nx) + 0.5) / nx)[None, None, :])
    T0 = 80.0 + mode
    mu = 1.0 - c["k"] * c["cz"] - 4.0 * c["k"] * (
        c["cx"] * _sin2(kx, nx) + c["cy"] * _sin2(ky, ny) + c["cz2"] * _sin2(kz, nz))
    Tn = oracle.heat_run(T0, np.zeros((ny, nx)), n, c, oracle.BC_CLAMP)
    assert np.max(np.abs((Tn - 80.0) - mu ** n * mode)) <= 1e-11 * mu ** n + _AMB_FLOOR


def test_uniform_relaxation_with_source_2d(oracle):
    # Uniform T0 and uniform P = p: T^n = T* + (T0 - T*)(1 - k cz)^n with
    # T* = t_amb + p/cz.  Pins the source and ambient terms and their scale.
    c = oracle.HEAT_COEFFS_2D
    p, t0, n = 7e-4, 330.0, 1000
    T0 = np.full((9, 14), t0)
    Tn = oracle.heat_run(T0, np.full((9, 14), p), n, c, oracle.BC_CLAMP)
    ts = c["t_amb"] + p / c["cz"]
    expect = ts + (t0 - ts) * (1.0 - c["k"] * c["cz"]) ** n
    assert np.max(np.abs(Tn - expect)) <= 1e-12 * expect


def test_uniform_relaxation_3d_no_source(oracle):
    c = oracle.HEAT_COEFFS_3D
    T0 = np.full((5, 6, 7), 333.0)
    n = 500
    Tn = oracle.heat_run(T0, np.zeros((6, 7)), n, c, oracle.BC_CLAMP)
    expect = 80.0 + (333.0 - 80.0) * (1.0 - c["k"] * c["cz"]) ** n
    assert np.max(np.abs(Tn - expect)) <= 1e-12 * expect


@pytest.mark.parametrize("nz", [1, 4])
def test_heat_sum_conservation_and_layer0_source(oracle, nz):
    # cz = 0, clamp: the stencil moves heat but never creates it, so
    # sum(T^n) = sum(T^0) + n*k*sum(P); in 3D P acts on layer 0 only.
    c = dict(ASYM, cz=0.0)
    T0, P = gs_inputs.heat_fields(15, 11, nz, seed=3)
    n = 200
    Tn = oracle.heat_run(T0, np.zeros_like(P, dtype=np.float64), n, c, oracle.BC_CLAMP)
    s0 = float(np.sum(T0.astype(np.float64)))
    assert abs(float(np.sum(Tn)) - s0) <= 1e-12 * s0
    Tp = oracle.heat_run(T0, P, n, c, oracle.BC_CLAMP)
    gain = n * c["k"] * float(np.sum(P.astype(np.float64)))
    assert abs(float(np.sum(Tp)) - s0 - gain) <= 1e-11 * s0


@pytest.mark.parametrize("nz", [1, 3])
def test_max_principle(oracle, nz):
    # With k(2cx+2cy+cz[+2cz2]) <= 1 every update is a convex combination of
    # neighbours and t_amb, plus k*P: bounds hold step by step.
    c = oracle.HEAT_COEFFS_2D if nz == 1 else oracle.HEAT_COEFFS_3D
    T, P = gs_inputs.heat_fields(13, 9, nz, seed=5)
    T = T.astype(np.float64)
    Pd = P.astype(np.float64)
    for _ in range(30):
        lo = min(T.min(), c["t_amb"])
        hi = max(T.max(), c["t_amb"])
        T = oracle.heat_run(T, Pd, 1, c, oracle.BC_CLAMP)
        assert T.min() >= lo - 1e-12 * hi
        assert T.max() <= hi + c["k"] * Pd.max() + 1e-12 * hi


def _heat_matrix(nx, ny, nz, c, bc):
    """Assemble T^{n+1} = A T^n + b cell by cell from the stencil's weights."""
    n = nx * ny * nz
    A = np.zeros((n, n))
    b = np.zeros(n)
    k = c["k"]
    dirs = [((1, 0, 0), c["cx"]), ((-1, 0, 0), c["cx"]), ((0, 1, 0), c["cy"]), ((0, -1, 0), c["cy"])]
    if nz > 1:
        dirs += [((0, 0, 1), c["cz2"]), ((0, 0, -1), c["cz2"])]

    def idx(x, y, z):
        return (z * ny + y) * nx + x

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = idx(x, y, z)
                A[i, i] += 1.0 - k * c["cz"]
                b[i] += k * c["cz"] * c["t_amb"]
                for (dx, dy, dz), w in dirs:
                    A[i, i] -= k * w
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz:
                        A[i, idx(xx, yy, zz)] += k * w
                    elif bc == 0:  # clamp: the missing neighbour is the cell itself
                        A[i, i] += k * w
    return A, b


@pytest.mark.parametrize("shape", [(5, 4, 1), (3, 4, 2)])
@pytest.mark.parametrize("bc", [0, 1])
def test_brute_force_matrix_power(oracle, shape, bc):
    nx, ny, nz = shape
    c = dict(k=0.5, cx=0.1, cy=0.13, cz=0.01, cz2=0.07, t_amb=80.0)
    T0, P = gs_inputs.heat_fields(nx, ny, nz, seed=11)
    A, b = _heat_matrix(nx, ny, nz, c, bc)
    src = np.zeros(nx * ny * nz)
    src[: nx * ny] = c["k"] * P.astype(np.float64).ravel()  # layer 0 (the only layer in 2D)
    b = b + src
    n = 7
    t = T0.astype(np.float64).ravel()
    expect = np.linalg.matrix_power(A, n) @ t + sum(np.linalg.matrix_power(A, j) for j in range(n)) @ b
    got = oracle.heat_run(T0, P, n, c, bc).ravel()
    assert np.max(np.abs(got - expect)) <= 1e-12 * np.max(np.abs(expect))


def test_zero_steps_and_degenerate_shapes(oracle):
    T0, P = gs_inputs.heat_fields(7, 1, 1, seed=2)  # a single row
    assert np.array_equal(oracle.heat_run(T0, P, 0, oracle.HEAT_COEFFS_2D), T0.astype(np.float64))
    # a 1x1 grid under clamp: every neighbour is the cell, only P and ambient act
    c = oracle.HEAT_COEFFS_2D
    T = oracle.heat_run(np.array([[330.0]]), np.array([[1e-3]]), 3, c)
    t = 330.0
    for _ in range(3):
        t = t + c["k"] * (1e-3 + c["cz"] * (c["t_amb"] - t))
    assert abs(T[0, 0] - t) <= 1e-12 * t
