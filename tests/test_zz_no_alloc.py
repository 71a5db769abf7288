"""gs_multi_step_noalloc, the fused multi-instance step for callers that
cannot call cudaMalloc (their device memory comes from their own allocator
or a fixed budget, or their loop cannot afford cudaMalloc's implicit device
synchronisation).  It must give the same results as the existing entry
point, gs_multi_step in GS_MULTI_FUSED mode, on two calls in a row: the
second call runs on the table the first one left behind.

Kept in a file of its own, collected after every other test file."""
import ctypes

import numpy as np
import pytest

import gs_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_09398_gb300  # noqa: F401


DIMS = [(130, 17), (5, 9), (64, 64), (200, 3), (1, 1), (77, 120), (300, 40)]


def _reference(fields_np, calls, stream):
    """The existing entry point: gs_multi_step(FUSED) with the same calls;
    returns the dense fields after each call."""
    import paper_2501_09398_gb300 as g

    nx = [d[0] for d in DIMS]
    ny = [d[1] for d in DIMS]
    m = g.gs_multi_create(nx, ny, g.GS_F32, g.GS_BC_CLAMP, stream.cuda_stream)
    bufs = g.MultiFields(m, nx, ny)
    out = []
    try:
        for i, (T, P) in enumerate(fields_np):
            g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
        for n in calls:
            g.gs_multi_step(m, n, 0, g.GS_MULTI_FUSED)
            out.append([g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T))
                        for i, (T, _) in enumerate(fields_np)])
    finally:
        g.gs_multi_destroy(m)
        del bufs
    return out


def test_noalloc_matches_fused_entry_point_on_two_calls():
    import torch

    import paper_2501_09398_gb300 as g

    stream = torch.cuda.Stream()
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=500 + i) for i, (w, h) in enumerate(DIMS)]
    calls = (9, 6)
    ref = _reference(fields_np, calls, stream)

    # caller-owned buffers: T0 holds the state, T1 the other half of the pair
    inst, keep = [], []
    for (w, h), (T, P) in zip(DIMS, fields_np):
        pitch = g.gs_required_pitch(g.GS_F32, w)
        t0 = torch.zeros((h, pitch), dtype=torch.float32, device="cuda")
        t1 = torch.zeros((h, pitch), dtype=torch.float32, device="cuda")
        p = torch.zeros((h, pitch), dtype=torch.float32, device="cuda")
        t0[:, :w] = torch.from_numpy(T).cuda()
        p[:, :w] = torch.from_numpy(P).cuda()
        keep.append((t0, t1, p))
        inst.append(dict(T0=t0.data_ptr(), T1=t1.data_ptr(), P=p.data_ptr(), nx=w, ny=h, pitch=pitch,
                         p_pitch=pitch))
    torch.cuda.synchronize()
    parity = 0
    for call, n in enumerate(calls):
        parity = g.gs_multi_step_noalloc(inst, parity, n, stream=stream.cuda_stream)
        assert parity == sum(calls[:call + 1]) % 2
        stream.synchronize()
        for i, ((w, h), bufs) in enumerate(zip(DIMS, keep)):
            got = bufs[parity][:, :w].cpu().numpy()
            assert np.array_equal(got, ref[call][i]), (call, i)


def test_noalloc_rejects_more_instances_than_its_table():
    import paper_2501_09398_gb300 as g

    n = g.GS_NOALLOC_MAX_INSTANCES + 1
    arr = (g.gs_instance * n)()
    c = g.gs_heat_coeffs(0.5, 0.1, 0.1, 0.01, 0.05, 80.0)
    out = ctypes.c_int32(0)
    st = g.raw_call("gs_multi_step_noalloc", arr, n, 0, 1, ctypes.byref(c), g.GS_F32, g.GS_BC_CLAMP, None,
                    ctypes.byref(out))
    assert st == g.GS_ERR_INVALID_ARG
    assert "257" in g.gs_last_error(None) and "256" in g.gs_last_error(None)
