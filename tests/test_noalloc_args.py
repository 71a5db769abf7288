"""gs_multi_step_noalloc and gs_multi_create refuse bad arguments before any
CUDA call (CPU).

Each case carries at least one invalid argument, so the call returns from
its checks and never reaches the device: the pointers below are
placeholders that nothing dereferences."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300

    return paper_2501_09398_gb300


FAKE = 0x100000  # 16-byte aligned, never dereferenced
GAP = 0x4000      # 16 KiB between placeholder buffers: an f32 64 x 32 field needs 8 KiB


def _inst(g, base=FAKE, **over):
    d = dict(T0=base, T1=base + GAP, P=base + 2 * GAP, nx=64, ny=32, pitch=64, p_pitch=64)
    d.update(over)
    return g.gs_instance(ctypes.c_void_p(d["T0"]), ctypes.c_void_p(d["T1"]), ctypes.c_void_p(d["P"]), d["nx"],
                         d["ny"], d["pitch"], d["p_pitch"])


def _call(g, insts, n=None, parity=0, n_iters=10, coeffs=None, storage=None, bc=None):
    arr = (g.gs_instance * max(1, len(insts)))(*insts)
    c = coeffs or g.gs_heat_coeffs(0.5, 0.1, 0.1, 0.01, 0.05, 80.0)
    out = ctypes.c_int32(-1)
    st = g._lib.gs_multi_step_noalloc(arr, len(insts) if n is None else n, parity, n_iters, ctypes.byref(c),
                                      g.GS_F32 if storage is None else storage,
                                      g.GS_BC_CLAMP if bc is None else bc, None, ctypes.byref(out))
    return st, g.gs_last_error(None), out.value


def test_instance_count_outside_the_table(g):
    for n in (0, -1, g.GS_NOALLOC_MAX_INSTANCES + 1):
        st, msg, out = _call(g, [_inst(g, nx=0)], n=n)  # nx = 0 too: invalid whatever is checked first
        assert st == g.GS_ERR_INVALID_ARG and out == -1
        assert "n_inst" in msg or "nx" in msg
    st, msg, _ = _call(g, [_inst(g)], n=0)
    assert st == g.GS_ERR_INVALID_ARG and str(g.GS_NOALLOC_MAX_INSTANCES) in msg


@pytest.mark.parametrize("kw,status", [
    (dict(parity=2), "INVALID_ARG"),
    (dict(n_iters=-1), "INVALID_ARG"),
    (dict(storage=7), "INVALID_ARG"),
    (dict(bc=2), "INVALID_ARG"),  # PEC is an FDTD boundary
])
def test_call_arguments(g, kw, status):
    st, _, out = _call(g, [_inst(g, nx=0)], **kw)  # a bad instance as a backstop
    assert st == getattr(g, "GS_ERR_" + status) and out == -1


def test_non_finite_coefficient(g):
    for k in ("k", "cx", "cz2", "t_amb"):
        c = g.gs_heat_coeffs(0.5, 0.1, 0.1, 0.01, 0.05, 80.0)
        setattr(c, k, float("nan"))
        st, msg, _ = _call(g, [_inst(g, nx=0)], coeffs=c)
        assert st == g.GS_ERR_NUMERIC, k


@pytest.mark.parametrize("over,storage", [
    (dict(T0=0), None),                  # NULL buffer
    (dict(T1=FAKE + 4), None),           # misaligned
    (dict(P=FAKE + 8), None),
    (dict(nx=0), None),
    (dict(ny=(1 << 20) + 1), None),
    (dict(pitch=63), None),              # below nx
    (dict(pitch=66), None),              # not a multiple of 16 bytes (f32: 4 elements)
    (dict(nx=60, pitch=60, p_pitch=60), 1),   # bf16 rows need 8-element pitches
    (dict(p_pitch=32), None),
])
def test_bad_instance_is_named(g, over, storage):
    # the second instance is the bad one; the message names it
    st, msg, out = _call(g, [_inst(g), _inst(g, **over)], storage=storage)
    assert st == g.GS_ERR_INVALID_ARG and out == -1
    assert "instance 1" in msg, msg


def test_null_arguments(g):
    c = g.gs_heat_coeffs(0.5, 0.1, 0.1, 0.01, 0.05, 80.0)
    assert g._lib.gs_multi_step_noalloc(None, 1, 0, 1, ctypes.byref(c), g.GS_F32, g.GS_BC_CLAMP, None,
                                        None) == g.GS_ERR_INVALID_ARG
    arr = (g.gs_instance * 1)(_inst(g, nx=0))
    assert g._lib.gs_multi_step_noalloc(arr, 1, 0, 1, None, g.GS_F32, g.GS_BC_CLAMP, None,
                                        None) == g.GS_ERR_INVALID_ARG


def test_multi_create_refusals_carry_a_message(g):
    # gs_multi_create's argument checks run before any CUDA call; each
    # refusal sets *out to NULL and leaves its reason in gs_last_error(NULL)
    i64 = ctypes.c_int64
    good = (i64 * 2)(64, 32)
    cases = [
        (2, (i64 * 2)(64, 0), g.GS_F32, g.GS_BC_CLAMP, "instance 1"),
        (2, (i64 * 2)(64, 1 << 21), g.GS_F32, g.GS_BC_CLAMP, "instance 1"),
        (2, good, 9, g.GS_BC_CLAMP, "dtype"),
        (2, good, g.GS_F32, g.GS_BC_PEC, "bc"),
        (0, good, g.GS_F32, g.GS_BC_CLAMP, "n < 1"),
    ]
    for n, ny, dt, bc, text in cases:
        h = ctypes.c_void_p(123)
        st = g._lib.gs_multi_create(ctypes.byref(h), n, good, ny, dt, bc, None)
        assert st == g.GS_ERR_INVALID_ARG and h.value is None, text
        assert text in g.gs_last_error(None), (text, g.gs_last_error(None))
    h = ctypes.c_void_p(123)
    assert g._lib.gs_multi_create(ctypes.byref(h), 2, None, good, g.GS_F32, g.GS_BC_CLAMP, None) \
        == g.GS_ERR_INVALID_ARG
    assert h.value is None


def test_overlapping_buffers_are_refused(g):
    # an instance whose T0 is its T1 would be updated in place while read
    st, msg, out = _call(g, [_inst(g, T1=FAKE)])
    assert st == g.GS_ERR_INVALID_ARG and out == -1
    assert "instance 0" in msg and "overlap" in msg, msg
    # instance 1's T1 starts inside instance 0's T0 (ny * pitch * 4 bytes long)
    b1 = FAKE + 0x100000
    st, msg, _ = _call(g, [_inst(g), _inst(g, base=b1, T1=FAKE + 0x1000)])
    assert st == g.GS_ERR_INVALID_ARG and "instances 0 and 1" in msg, msg
    # a power map that overlaps another instance's T buffer
    st, msg, _ = _call(g, [_inst(g), _inst(g, base=b1, P=FAKE + GAP)])
    assert st == g.GS_ERR_INVALID_ARG and "overlap" in msg, msg
    # the last row's padding counts: T1 starting one element before T0's end
    st, msg, _ = _call(g, [_inst(g, T1=FAKE + 32 * 64 * 4 - 4 * 4)])
    assert st == g.GS_ERR_INVALID_ARG and "overlap" in msg, msg


def test_shared_power_map_is_accepted(g):
    # P buffers are only read, so instances may share one; n_iters = 0 runs
    # every check and returns before any CUDA call
    b1 = FAKE + 0x100000
    st, msg, out = _call(g, [_inst(g), _inst(g, base=b1, P=FAKE + 2 * GAP)], parity=1, n_iters=0)
    assert st == g.GS_OK, msg
    assert out == 1
    # adjacent (touching, not overlapping) buffers are fine too
    st, msg, _ = _call(g, [_inst(g, T1=FAKE + 32 * 64 * 4)], n_iters=0)
    assert st == g.GS_OK, msg
