"""mmlttb_minmaxlttb_noalloc, the entry point for callers that cannot allocate
device memory (serving loops that forbid cudaMalloc/cudaFree because those can
synchronize the device, plugin hosts without an allocator): through the C ABI, two
calls in a row must return exactly the indices of the workspace entry point
mmlttb_minmaxlttb with a clean status word (mmlttb_noalloc_status), and sizes
beyond its static scratch must be refused.  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

_vp, _i64, _i32, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int


def noalloc_fn(mm):
    f = mm.lib.mmlttb_minmaxlttb_noalloc
    f.restype = _int
    f.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _i32, _int, _vp, _i64, _vp, _vp]
    return f


def noalloc_status(mm):
    f = mm.lib.mmlttb_noalloc_status
    f.restype = _int
    f.argtypes = [_vp, _vp]
    v = ctypes.c_int(-1)
    rc = f(ctypes.byref(v), torch.cuda.current_stream().cuda_stream)
    assert rc == mm.OK, mm.strerror(rc)
    return v.value


def call_noalloc(mm, y, n_out, r_ps, x=None, binmode=0):
    n = y.numel()
    cap = max(min(n, n_out), 1)
    out = torch.full((cap,), -1, dtype=torch.int64, device=y.device)
    cnt = torch.full((1,), -1, dtype=torch.int64, device=y.device)
    yd = mm.F32 if y.dtype == torch.float32 else mm.F64
    xk = mm.X_IMPLICIT if x is None else (mm.X_I64 if x.dtype == torch.int64 else mm.X_F64)
    rc = noalloc_fn(mm)(y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out,
                        r_ps, binmode, out.data_ptr(), cap, cnt.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
    return rc, out, cnt


def cases():
    y1 = torch.from_numpy(synth.random_walk(1_000_000, seed=0, dtype=np.float32)).cuda()
    y2 = torch.from_numpy(synth.random_walk(300_000, seed=1, dtype=np.float64)).cuda()
    x2 = torch.from_numpy(synth.exp_gaps_x(300_000, seed=1, mean_gap=50.0, big_gaps=3, big_gap=10**7)).cuda()
    y3 = torch.from_numpy(synth.random_walk(200_000, seed=2, dtype=np.float32)).cuda()
    y4 = torch.from_numpy(synth.random_walk(10_000_000, seed=4, dtype=np.float32)).cuda()
    return [
        (y1, 1000, 4, None, 0),     # MinMax preselection + transition-table LTTB
        (y4, 1000, 4, None, 0),     # y above 8 MiB: streaming kernel, then the fused tail
        (y2, 2000, 4, x2, 1),       # x-width bins, float64 y
        (y3, 60_000, 4, None, 0),   # r_ps * n_out >= n: LTTB on all points
        (y3, 40, 64, None, 0),      # large preselected buckets: grid-wide LTTB
        (y3, 300_000, 4, None, 0),  # n_out >= n: every index
    ]


def test_noalloc_equals_workspace_entry_point_twice(mm):
    for y, n_out, r_ps, x, bm in cases():
        exp = mm.minmaxlttb(y, n_out, r_ps, x=x, binmode=bm)
        for _ in range(2):  # the second call reuses scratch left by the first
            rc, out, cnt = call_noalloc(mm, y, n_out, r_ps, x, bm)
            assert rc == mm.OK, mm.strerror(rc)
            assert noalloc_status(mm) == 0
            torch.cuda.synchronize()
            k = int(cnt.item())
            assert k == exp.numel()
            assert torch.equal(out[:k], exp), (y.numel(), n_out, r_ps)


def test_noalloc_refuses_sizes_beyond_its_scratch(mm):
    y = torch.from_numpy(synth.random_walk(5_000_000, seed=3, dtype=np.float32)).cuda()
    rc, out, cnt = call_noalloc(mm, y, 200_000, 4)  # 400 000 bins: far above 4 MiB
    assert rc == mm.ESCRATCH
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1 and bool((out == -1).all())


def test_noalloc_status_rejects_a_null_pointer(mm):
    f = mm.lib.mmlttb_noalloc_status
    f.restype = _int
    f.argtypes = [_vp, _vp]
    assert f(None, torch.cuda.current_stream().cuda_stream) == mm.EINVAL
