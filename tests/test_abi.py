"""C-ABI contract checks that need no GPU: the library builds and loads, it
exports every function include/*.h declares, and argument validation that
happens before any CUDA call returns the documented status codes."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(gs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_api():
    names = _declared()
    for core in ("gs_create", "gs_destroy", "gs_step", "gs_graph_build", "gs_graph_launch", "gs_graph_destroy",
                 "gs_read_field", "gs_upload", "gs_bind_field", "gs_set_heat_coeffs", "gs_set_fdtd_params"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings_and_pitch(lib):
    import paper_2501_09398_gb300 as g

    assert g.gs_status_string(g.GS_OK) == "GS_OK"
    assert g.gs_status_string(g.GS_ERR_TIMEOUT) == "GS_ERR_TIMEOUT"
    assert g.gs_required_pitch(g.GS_F32, 1) == 4
    assert g.gs_required_pitch(g.GS_F32, 129) == 132
    assert g.gs_required_pitch(g.GS_BF16, 129) == 136
    assert g.gs_required_pitch(g.GS_F16, 512) == 512
    out = ctypes.c_int64()
    assert g.raw_call("gs_required_pitch", g.GS_F32, 0, ctypes.byref(out)) == g.GS_ERR_INVALID_ARG
    assert g.raw_call("gs_required_pitch", 9, 4, ctypes.byref(out)) == g.GS_ERR_INVALID_ARG


@pytest.mark.parametrize("args", [
    (0, 0, 16, 1),          # nx = 0
    (0, 16, 16, 2),         # 2D with nz != 1
    (2, 16, 16, 15),        # FDTD not cubic
    (7, 16, 16, 1),         # unknown kind
    (0, 1 << 21, 1, 1),     # too large
])
def test_create_rejects_bad_arguments(lib, args):
    import paper_2501_09398_gb300 as g

    kind, nx, ny, nz = args
    h = ctypes.c_void_p()
    st = g.raw_call("gs_create", ctypes.byref(h), kind, nx, ny, nz, g.GS_F32, g.GS_BC_CLAMP, None)
    assert st == g.GS_ERR_INVALID_ARG
    assert h.value is None
    assert g.gs_last_error(None)


def test_create_rejects_wrong_boundary(lib):
    import paper_2501_09398_gb300 as g

    h = ctypes.c_void_p()
    assert g.raw_call("gs_create", ctypes.byref(h), g.GS_FDTD3D, 8, 8, 8, g.GS_F32, g.GS_BC_CLAMP, None) \
        == g.GS_ERR_INVALID_ARG
    assert g.raw_call("gs_create", ctypes.byref(h), g.GS_HEAT2D, 8, 8, 1, g.GS_F32, g.GS_BC_PEC, None) \
        == g.GS_ERR_INVALID_ARG
    assert g.raw_call("gs_destroy", None) == g.GS_OK


def test_null_handles(lib):
    import paper_2501_09398_gb300 as g

    assert g.raw_call("gs_step", None, 1, 1) == g.GS_ERR_INVALID_ARG
    assert g.raw_call("gs_sync", None) == g.GS_ERR_INVALID_ARG
    assert g.raw_call("gs_graph_launch", None, 1) == g.GS_ERR_INVALID_ARG


def test_null_handle_refusals_leave_a_message(lib):
    # with no context to hold it, the reason goes to gs_last_error(NULL)
    import paper_2501_09398_gb300 as g

    out64 = ctypes.c_int64()
    out32 = ctypes.c_int32()
    cases = [
        ("gs_step", (None, 1, 1)), ("gs_sync", (None,)), ("gs_graph_build", (None, 10)),
        ("gs_graph_launch", (None, 1)), ("gs_graph_destroy", (None,)), ("gs_set_scale", (None, 1.0)),
        ("gs_bind_field", (None, g.GS_FIELD_T0, None, 16)), ("gs_get_time", (None, ctypes.byref(out64))),
        ("gs_get_parity", (None, ctypes.byref(out32))), ("gs_get_plan", (None, ctypes.byref(g.gs_plan()))),
        ("gs_get_stats", (None, ctypes.byref(g.gs_stats()))), ("gs_set_fdtd_media", (None, None, 0)),
        ("gs_required_pitch", (g.GS_F32, 0, ctypes.byref(out64))),
        ("gs_multi_sync", (None,)), ("gs_multi_get_parity", (None, ctypes.byref(out32))),
        ("gs_multi_get_stats", (None, ctypes.byref(g.gs_stats()))),
        ("gs_multi_set_plan", (None, ctypes.byref(g.gs_multi_plan()))),
        ("gs_multi_set_heat_coeffs", (None, None)),
        ("gs_model_total", (None, 10.0, ctypes.byref(ctypes.c_double()))),
    ]
    h = ctypes.c_void_p()
    for name, args in cases:
        # a known message first (gs_create refusing an unknown kind), which
        # the refusal under test must replace with its own
        g.raw_call("gs_create", ctypes.byref(h), 7, 8, 8, 1, g.GS_F32, g.GS_BC_CLAMP, None)
        assert g.gs_last_error(None) == "unknown kind"
        assert g.raw_call(name, *args) == g.GS_ERR_INVALID_ARG, name
        assert g.gs_last_error(None) not in ("", "unknown kind"), name
