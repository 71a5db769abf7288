"""gs_multi_step_noalloc, the fused multi-instance step for callers that
cannot call cudaMalloc (their device memory comes from their own allocator
or a fixed budget, or their loop cannot afford cudaMalloc's implicit device
synchronisation).  It must give the same results as the existing entry
point, gs_multi_step in GS_MULTI_FUSED mode, on calls in a row: each later
call runs on the table the one before it left behind, including a call with
fewer instances than the one before.  It must also leave the device's free
memory unchanged.

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
SUBSET = [0, 2, 5]  # the instances of the smaller later call


def _reference(dims, states, calls, stream, dtype, bc):
    """The existing entry point: gs_multi_step(FUSED) from the given dense
    states with the same calls; returns the dense fields after each call and
    the stored (rounded) initial states."""
    import paper_2501_09398_gb300 as g

    nx = [d[0] for d in dims]
    ny = [d[1] for d in dims]
    m = g.gs_multi_create(nx, ny, dtype, bc, stream.cuda_stream)
    bufs = g.MultiFields(m, nx, ny, dtype)
    out = []
    try:
        for i, (T, P) in enumerate(states):
            g.gs_multi_upload(m, i, g.GS_FIELD_T, T)
            g.gs_multi_upload(m, i, g.GS_FIELD_P, P)
        stored = [(g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T)),
                   g.gs_multi_read_field(m, i, g.GS_FIELD_P, np.empty_like(P))) for i, (T, P) in enumerate(states)]
        for n in calls:
            g.gs_multi_step(m, n, 0, g.GS_MULTI_FUSED)
            out.append([g.gs_multi_read_field(m, i, g.GS_FIELD_T, np.empty_like(T))
                        for i, (T, _) in enumerate(states)])
    finally:
        g.gs_multi_destroy(m)
        del bufs
    return out, stored


def _caller_buffers(states, dtype):
    """Caller-owned buffers (torch tensors) holding the stored initial states
    in T0 and the power maps in P; values are exactly representable in the
    storage type (they were read back from it)."""
    import torch

    import paper_2501_09398_gb300 as g

    tdt = {g.GS_F32: torch.float32, g.GS_BF16: torch.bfloat16, g.GS_F16: torch.float16}[dtype]
    inst, keep = [], []
    for T, P in states:
        h, w = T.shape
        pitch = g.gs_required_pitch(dtype, w)
        t0 = torch.zeros((h, pitch), dtype=tdt, device="cuda")
        t1 = torch.zeros((h, pitch), dtype=tdt, device="cuda")
        p = torch.zeros((h, pitch), dtype=tdt, device="cuda")
        t0[:, :w] = torch.from_numpy(T).to(tdt).cuda()
        p[:, :w] = torch.from_numpy(P).to(tdt).cuda()
        keep.append((t0, t1, p))
        inst.append(dict(T0=t0.data_ptr(), T1=t1.data_ptr(), P=p.data_ptr(), nx=w, ny=h, pitch=pitch,
                         p_pitch=pitch))
    torch.cuda.synchronize()
    return inst, keep


def _dense(buf, w):
    return buf[:, :w].float().cpu().numpy()


@pytest.mark.parametrize("dtype_name,bc", [("f32", 0), ("bf16", 0), ("f16", 0), ("f32", 1), ("f16", 1)])
def test_noalloc_matches_fused_entry_point_on_calls_in_a_row(dtype_name, bc):
    import torch

    import paper_2501_09398_gb300 as g

    dtype = g.DTYPES[dtype_name]
    coeffs = dict(k=0.5, cx=0.1, cy=0.1, cz=0.01, cz2=0.05, t_amb=80.0)
    stream = torch.cuda.Stream()
    fields_np = [gs_inputs.heat_fields(w, h, 1, seed=500 + i) for i, (w, h) in enumerate(DIMS)]
    calls = (9, 6)
    ref, stored = _reference(DIMS, fields_np, calls, stream, dtype, bc)
    inst, keep = _caller_buffers(stored, dtype)

    parity = 0
    for call, n in enumerate(calls):
        parity = g.gs_multi_step_noalloc(inst, parity, n, coeffs=coeffs, dtype=dtype, bc=bc,
                                         stream=stream.cuda_stream)
        assert parity == sum(calls[:call + 1]) % 2
        stream.synchronize()
        for i, ((w, h), bufs) in enumerate(zip(DIMS, keep)):
            assert np.array_equal(_dense(bufs[parity], w), ref[call][i]), (call, i)

    # a smaller batch next: the table still holds the larger batch's rows
    # past the subset's, which the call must not read
    before = [[_dense(b, w) for b in bufs[:2]] for (w, _), bufs in zip(DIMS, keep)]
    sub_dims = [DIMS[i] for i in SUBSET]
    sub_states = [(ref[-1][i], stored[i][1]) for i in SUBSET]
    sub_ref, _ = _reference(sub_dims, sub_states, (4,), stream, dtype, bc)
    p2 = g.gs_multi_step_noalloc([inst[i] for i in SUBSET], parity, 4, coeffs=coeffs, dtype=dtype, bc=bc,
                                 stream=stream.cuda_stream)
    stream.synchronize()
    assert p2 == parity
    for k, i in enumerate(SUBSET):
        assert np.array_equal(_dense(keep[i][p2], DIMS[i][0]), sub_ref[0][k]), ("subset", i)
    for i, ((w, _), bufs) in enumerate(zip(DIMS, keep)):
        if i not in SUBSET:
            for b in range(2):
                assert np.array_equal(_dense(bufs[b], w), before[i][b]), ("untouched", i, b)


def test_noalloc_leaves_free_device_memory_unchanged():
    import torch

    import paper_2501_09398_gb300 as g

    stream = torch.cuda.Stream()
    states = [gs_inputs.heat_fields(w, h, 1, seed=900 + i) for i, (w, h) in enumerate(DIMS)]
    inst, keep = _caller_buffers(states, g.GS_F32)
    parity = g.gs_multi_step_noalloc(inst, 0, 3, stream=stream.cuda_stream)  # set-up happens here at the latest
    stream.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(10):
        parity = g.gs_multi_step_noalloc(inst, parity, 5, stream=stream.cuda_stream)
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    del keep


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
