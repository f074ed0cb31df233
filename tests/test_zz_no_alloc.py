"""isycos_mi_windows_noalloc: window MI for callers that cannot allocate device memory (GPU).

Callers under a runtime that owns all device memory, or in loops where cudaMalloc would
synchronise the device, use this entry point: it takes its work memory from a static device
array instead of allocating.  Its results must equal those of the context path
(isycos_mi_windows) -- integer sums exactly, scalars within the 1e-12 used by the other
parity tests -- on two calls in a row, since the second call reuses the scratch the first
one left behind.  Invalid windows come back as NaN with zero sums, and a warmed call leaves
the device's free memory unchanged.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2204_09131_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _windows(rng, n, count):
    sizes = np.concatenate([[5, 31, 32, 33, 64, 65, 128, 129, 4096, 4097, 8192],
                            rng.integers(5, 3000, count)]).astype(np.int32)
    starts = np.array([int(rng.integers(0, n - m + 1)) for m in sizes], dtype=np.int64)
    return starts, sizes


def _call(L, dx, dy, n, starts, sizes, k, max_m, stream):
    import torch
    d_starts = torch.from_numpy(starts).cuda()
    d_sizes = torch.from_numpy(sizes).cuda()
    d_out = torch.zeros(len(sizes) * 40, dtype=torch.uint8, device="cuda")
    stream.synchronize()
    st = L.isycos_mi_windows_noalloc(dx.data_ptr(), dy.data_ptr(), n, d_starts.data_ptr(),
                                     d_sizes.data_ptr(), len(sizes), k, max_m,
                                     d_out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return st, d_out


def test_noalloc_matches_the_context_path_on_two_calls():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api

    n = 40000
    x, y, _ = synth.planted_pair(6, 0, n)
    rng = np.random.default_rng(12)
    calls = [_windows(rng, n, 700), _windows(rng, n, 300)]

    # reference results through the context path
    refs = []
    with api.Context(0) as ctx:
        xs = api.isycos_put_series(ctx, x)
        ys = api.isycos_put_series(ctx, y)
        for starts, sizes in calls:
            refs.append(api.isycos_mi_windows(ctx, api.windows_array(xs, ys, starts, sizes), 4))

    L = api.lib()
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y).cuda()
    stream = torch.cuda.current_stream()
    for (starts, sizes), ref in zip(calls, refs):
        st, d_out = _call(L, dx, dy, n, starts, sizes, 4, int(sizes.max()), stream)
        assert st == api.OK
        got = d_out.cpu().numpy().view(api.MI_OUT_DTYPE)
        assert np.array_equal(got["s_psi"], ref["s_psi"])
        assert np.array_equal(got["s_log"], ref["s_log"])
        assert np.max(np.abs(got["mi"] - ref["mi"])) <= TOL
        assert np.max(np.abs(got["nmi"] - ref["nmi"])) <= TOL

    # invalid windows (past the end, before the start, fewer than k + 1 points, above max_m)
    # come back as NaN with zero sums; the valid windows around them are unaffected
    starts, sizes = calls[1]
    bad_starts = np.concatenate([starts[:4], [n - 10, -1, 100, 200]]).astype(np.int64)
    bad_sizes = np.concatenate([sizes[:4], [64, 32, 4, 3000]]).astype(np.int32)
    st, d_out = _call(L, dx, dy, n, bad_starts, bad_sizes, 4, 2048, stream)
    assert st == api.OK
    got = d_out.cpu().numpy().view(api.MI_OUT_DTYPE)
    assert np.array_equal(got["s_psi"][:4], refs[1]["s_psi"][:4])
    assert np.array_equal(got["mi"][:4], refs[1]["mi"][:4])
    for f in ("mi", "h_w", "nmi"):
        assert np.all(np.isnan(got[f][4:])), f
    assert np.all(got["s_psi"][4:] == 0) and np.all(got["s_log"][4:] == 0)

    # a warmed call takes no device memory: the free memory is the same before and after
    starts, sizes = calls[0]
    d_starts = torch.from_numpy(starts).cuda()
    d_sizes = torch.from_numpy(sizes).cuda()
    d_out = torch.zeros(len(sizes) * 40, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = L.isycos_mi_windows_noalloc(dx.data_ptr(), dy.data_ptr(), n, d_starts.data_ptr(),
                                     d_sizes.data_ptr(), len(sizes), 4, int(sizes.max()),
                                     d_out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == api.OK and free1 == free0, (free0, free1)
    got = d_out.cpu().numpy().view(api.MI_OUT_DTYPE)
    assert np.array_equal(got["s_psi"], refs[0]["s_psi"])

    # sizes beyond the static scratch are rejected before any device work
    st = L.isycos_mi_windows_noalloc(dx.data_ptr(), dy.data_ptr(), n, None, None, 65537, 4, 64,
                                     None, stream.cuda_stream)
    assert st == api.E_INVAL
