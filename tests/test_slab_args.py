"""gs_slab_create refuses bad arguments before any CUDA call (CPU): each case
below carries an invalid argument, so the call returns from its checks and
never reaches a device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300

    return paper_2501_09398_gb300


@pytest.mark.parametrize("args,text", [
    ((3, 64, 64, 1, 0, 0, 2, 1), "kind"),                  # the skeleton has no slabs
    ((0, 64, 64, 1, 0, 0, 0, 1), "n_slabs"),
    ((0, 64, 64, 1, 0, 0, 65, 1), "n_slabs"),
    ((0, 64, 64, 1, 0, 0, 2, 0), "halo"),
    ((0, 64, 64, 1, 0, 0, 2, 5), "halo"),
    ((2, 32, 32, 32, 0, 2, 2, 2), "halo"),                 # FDTD halo is 1
    ((0, 64, 10, 1, 0, 0, 4, 3), "slabs of at least 3"),  # 2 rows a slab
    ((1, 64, 64, 7, 0, 0, 4, 2), "slabs of at least 2"),  # 3D: planes
    ((2, 8, 8, 8, 0, 2, 10, 1), "slabs of at least 1"),   # FDTD: 9 planes, 10 slabs
    ((2, 8, 8, 9, 0, 2, 2, 1), "cubic"),
    ((0, 64, 64, 2, 0, 0, 2, 1), "nz == 1"),
    ((0, 64, 64, 1, 0, 2, 2, 1), "bc"),                    # PEC on a thermal grid
    ((2, 8, 8, 8, 0, 0, 2, 1), "bc"),                      # clamp on FDTD
    ((0, 64, 64, 1, 5, 0, 2, 1), "dtype"),
])
def test_slab_create_refusals(g, args, text):
    kind, nx, ny, nz, dt, bc, n, halo = args
    h = ctypes.c_void_p(123)
    st = g._lib.gs_slab_create(ctypes.byref(h), kind, nx, ny, nz, dt, bc, n, halo, None)
    assert st == g.GS_ERR_INVALID_ARG and h.value is None
    assert text in g.gs_last_error(None), g.gs_last_error(None)


def test_null_handles(g):
    assert g._lib.gs_slab_create(None, 0, 8, 8, 1, 0, 0, 1, 1, None) == g.GS_ERR_INVALID_ARG
    assert g._lib.gs_slab_destroy(None) == g.GS_OK
    assert g._lib.gs_slab_step(None, 1, 0) == g.GS_ERR_INVALID_ARG
    a, b = ctypes.c_int64(), ctypes.c_int64()
    assert g._lib.gs_slab_extent(None, 0, ctypes.byref(a), ctypes.byref(b)) == g.GS_ERR_INVALID_ARG
    assert g.gs_slab_last_error(None) == ""
