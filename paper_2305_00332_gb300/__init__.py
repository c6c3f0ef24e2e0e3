"""GB300 (sm_103a) MinMaxLTTB: Python binding of libmmlttb.so.

MinMaxLTTB (arXiv 2305.00332, Sec. 3) = MinMax preselection (argmin/argmax of y
per bin, first and last point kept) followed by LTTB on the preselected points.
Every step runs in the CUDA library; this module only marshals arguments: torch
tensors in, device pointers and the current CUDA stream out to the C ABI declared
in include/mmlttb.h.  There is no CPU fallback: importing fails loudly when the
library has not been built (run __graft_entry__.build()).
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmmlttb.so")

OK, EINVAL, ENOSPC, ECUDA, ETIMEOUT, ERANGE, EDEVICE, ENOMEM, ESCRATCH = 0, -1, -2, -3, -4, -6, -7, -8, -9
F32, F64 = 0, 1
X_IMPLICIT, X_I64, X_F64 = 0, 1, 2
BINS_INDEX, BINS_XWIDTH = 0, 1
NAN_AWARE = 0x10
OP_PRESELECT, OP_LTTB, OP_MINMAXLTTB, OP_M4 = 0, 1, 2, 3
PATH_AUTO, PATH_SPLIT, PATH_FUSED_TAIL, PATH_FUSED = 0, 1, 2, 3

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

lib = ctypes.CDLL(LIB_PATH)

_i64, _i32, _vp, _sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t
_int = ctypes.c_int

lib.mmlttb_strerror.restype = ctypes.c_char_p
lib.mmlttb_strerror.argtypes = [_int]
lib.mmlttb_last_cuda_error.restype = _int
lib.mmlttb_version.restype = _int
lib.mmlttb_workspace_bytes.restype = _int
lib.mmlttb_workspace_bytes.argtypes = [_int, _int, _int, _i64, _i64, _i32, _int, ctypes.POINTER(_sz)]
lib.mmlttb_minmax_preselect.restype = _int
lib.mmlttb_minmax_preselect.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _i32, _int, _vp, _i64, _vp,
                                        _vp, _sz, _vp]
lib.mmlttb_lttb.restype = _int
lib.mmlttb_lttb.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _vp, _i64, _vp, _vp, _sz, _vp]
lib.mmlttb_minmaxlttb.restype = _int
lib.mmlttb_minmaxlttb.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _i32, _int, _vp, _i64, _vp, _vp,
                                  _sz, _vp]
lib.mmlttb_m4.restype = _int
lib.mmlttb_m4.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _int, _vp, _i64, _vp, _vp, _sz, _vp]
lib.mmlttb_workspace_status.restype = _int
lib.mmlttb_workspace_status.argtypes = [_vp, ctypes.POINTER(_int), _vp]
lib.mmlttb_host_buffer_bytes.restype = _int
lib.mmlttb_host_buffer_bytes.argtypes = [_int, _int, _i64, _i64, _i32, _int, ctypes.POINTER(_sz)]
lib.mmlttb_host_buffer_bytes_inplace.restype = _int
lib.mmlttb_host_buffer_bytes_inplace.argtypes = [_int, _int, _i64, _i64, _i32, _int, ctypes.POINTER(_sz)]
lib.mmlttb_minmaxlttb_host.restype = _int
lib.mmlttb_minmaxlttb_host.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _i32, _int, _vp, _i64, _vp,
                                       _vp, _sz, _vp]
lib.mmlttb_set_timing_events.restype = _int
lib.mmlttb_set_timing_events.argtypes = [_vp, _vp]
lib.mmlttb_launch_count.restype = ctypes.c_ulonglong
lib.mmlttb_stream_variant_info.restype = _int
lib.mmlttb_stream_variant_info.argtypes = [_int, ctypes.POINTER(_int), ctypes.POINTER(_int)]
lib.mmlttb_autotune.restype = _int
lib.mmlttb_autotune.argtypes = [_int, _vp, _i64, _i64, _i32, _vp, _i64, _vp, _sz, _vp, ctypes.POINTER(_int),
                                ctypes.POINTER(ctypes.c_float)]
lib.mmlttb_get_stream_variant.restype = _int
lib.mmlttb_get_stream_variant.argtypes = [_int, ctypes.POINTER(_int)]
lib.mmlttb_set_stream_variant.restype = _int
lib.mmlttb_set_stream_variant.argtypes = [_int, _int]
lib.mmlttb_set_stage_events.restype = _int
lib.mmlttb_set_stage_events.argtypes = [ctypes.POINTER(_vp), _int]


class MMLTTBError(RuntimeError):
    def __init__(self, code, where):
        msg = lib.mmlttb_strerror(code).decode()
        if code == ECUDA:
            msg += f" (cudaError {lib.mmlttb_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{code}]")
        self.code = code


def _check(code, where):
    if code != OK:
        raise MMLTTBError(code, where)


def strerror(code):
    return lib.mmlttb_strerror(code).decode()


def _ydt(y):
    if y.dtype == torch.float32:
        return F32
    if y.dtype == torch.float64:
        return F64
    raise TypeError(f"y must be float32 or float64, got {y.dtype}")


def _xkind(x):
    if x is None:
        return X_IMPLICIT
    if x.dtype == torch.int64:
        return X_I64
    if x.dtype == torch.float64:
        return X_F64
    raise TypeError(f"x must be int64 or float64, got {x.dtype}")


def _binmode(binmode, nan_aware=False):
    flag = NAN_AWARE if nan_aware else 0
    if isinstance(binmode, int) and binmode & NAN_AWARE:
        flag, binmode = NAN_AWARE, binmode & ~NAN_AWARE
    if binmode in (BINS_INDEX, "index"):
        return BINS_INDEX | flag
    if binmode in (BINS_XWIDTH, "xwidth", "x"):
        return BINS_XWIDTH | flag
    raise ValueError(f"unknown bin mode {binmode!r}")


def _check_inputs(y, x, cuda=True):
    if y.dim() != 1 or not y.is_contiguous():
        raise ValueError("y must be a contiguous 1-D tensor")
    if cuda and not y.is_cuda:
        raise ValueError("y must be a CUDA tensor (the kernels read device memory)")
    if x is not None:
        if x.dim() != 1 or not x.is_contiguous() or x.numel() != y.numel():
            raise ValueError("x must be a contiguous 1-D tensor of the same length as y")
        if x.device != y.device:
            raise ValueError("x and y must be on the same device")


def _on(t, device, name):
    """t must live on `device` (the kernels write or read it there)."""
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, not {t.device}")
    return t


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def workspace_bytes(op, ydtype, xkind, n_in, n_out, r_ps=2, binmode=BINS_INDEX):
    """Bytes of workspace `op` needs on the current device (mmlttb_workspace_bytes)."""
    b = ctypes.c_size_t(0)
    _check(lib.mmlttb_workspace_bytes(op, ydtype, xkind, n_in, n_out, r_ps, _binmode(binmode),
                                      ctypes.byref(b)), "mmlttb_workspace_bytes")
    return b.value


def _workspace(nbytes, device, workspace):
    if workspace is None:
        return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
    return _on(workspace, device, "workspace")  # the C ABI checks the size (MMLTTB_ENOSPC)


def _finish(out, count, sync):
    if not sync:
        return out, count
    return out[: int(count.item())]


def minmax_preselect(y, n_out, r_ps, x=None, binmode=BINS_INDEX, out=None, workspace=None, sync=True,
                     nan_aware=False):
    """MinMax preselection (mmlttb_minmax_preselect): int64 indices of point 0, the
    per-bin argmin/argmax of floor(n_out*r_ps/2) bins, and point n-1."""
    _check_inputs(y, x)
    n = y.numel()
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode, nan_aware)
    cap = min(n, (n_out * r_ps // 2) * 2 + 2)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
    _on(out, y.device, "out")
    count = torch.empty(1, dtype=torch.int64, device=y.device)
    ws = _workspace(workspace_bytes(OP_PRESELECT, yd, xk, n, n_out, r_ps, bm), y.device, workspace)
    _check(lib.mmlttb_minmax_preselect(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out, r_ps, bm,
        out.data_ptr(), out.numel(), count.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), _stream(y.device)),
        "mmlttb_minmax_preselect")
    return _finish(out, count, sync)


def m4(y, n_out, x=None, binmode=BINS_INDEX, out=None, workspace=None, sync=True, nan_aware=False):
    """M4 (mmlttb_m4): per bin of floor(n_out/4) bins over all points, the first,
    argmin, argmax and last index, sorted and without repeats."""
    _check_inputs(y, x)
    n = y.numel()
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode, nan_aware)
    cap = min(n, 4 * (n_out // 4))
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
    _on(out, y.device, "out")
    count = torch.empty(1, dtype=torch.int64, device=y.device)
    ws = _workspace(workspace_bytes(OP_M4, yd, xk, n, n_out, 4, bm), y.device, workspace)
    _check(lib.mmlttb_m4(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out, bm,
        out.data_ptr(), out.numel(), count.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(),
        _stream(y.device)), "mmlttb_m4")
    return _finish(out, count, sync)


def lttb(y, n_out, x=None, out=None, workspace=None, sync=True):
    """Plain LTTB on all points (mmlttb_lttb): min(n_out, n) int64 indices."""
    _check_inputs(y, x)
    n = y.numel()
    yd, xk = _ydt(y), _xkind(x)
    cap = min(n, n_out)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
    _on(out, y.device, "out")
    count = torch.empty(1, dtype=torch.int64, device=y.device)
    ws = _workspace(workspace_bytes(OP_LTTB, yd, xk, n, n_out), y.device, workspace)
    _check(lib.mmlttb_lttb(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out,
        out.data_ptr(), out.numel(), count.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), _stream(y.device)),
        "mmlttb_lttb")
    return _finish(out, count, sync)


def minmaxlttb(y, n_out, r_ps=4, x=None, binmode=BINS_INDEX, out=None, workspace=None, sync=True):
    """MinMaxLTTB (mmlttb_minmaxlttb): min(n_out, n) int64 indices (fewer when
    x-width bins leave fewer than n_out points preselected)."""
    _check_inputs(y, x)
    n = y.numel()
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode)
    cap = min(n, n_out)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
    _on(out, y.device, "out")
    count = torch.empty(1, dtype=torch.int64, device=y.device)
    ws = _workspace(workspace_bytes(OP_MINMAXLTTB, yd, xk, n, n_out, r_ps, bm), y.device, workspace)
    _check(lib.mmlttb_minmaxlttb(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out, r_ps, bm,
        out.data_ptr(), out.numel(), count.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), _stream(y.device)),
        "mmlttb_minmaxlttb")
    return _finish(out, count, sync)


def workspace_status(workspace):
    """Status word of a workspace after the calls that used it (blocking)."""
    if not workspace.is_cuda:
        raise ValueError("workspace must be a CUDA tensor")
    st = ctypes.c_int(0)
    _check(lib.mmlttb_workspace_status(workspace.data_ptr(), ctypes.byref(st), _stream(workspace.device)),
           "mmlttb_workspace_status")
    return st.value


def host_buffer_bytes(ydtype, xkind, n_in, n_out, r_ps=4, binmode=BINS_INDEX, inplace=False):
    """Device bytes mmlttb_minmaxlttb_host needs: output, workspace and a staged copy
    of the series (any host memory), or with inplace=True without the copy (pinned or
    registered inputs, read in place)."""
    b = ctypes.c_size_t(0)
    f = lib.mmlttb_host_buffer_bytes_inplace if inplace else lib.mmlttb_host_buffer_bytes
    _check(f(ydtype, xkind, n_in, n_out, r_ps, _binmode(binmode), ctypes.byref(b)), "mmlttb_host_buffer_bytes")
    return b.value


def minmaxlttb_host(y, n_out, r_ps=4, x=None, binmode=BINS_INDEX, out=None, device_buffer=None,
                    device=None):
    """MinMaxLTTB on host tensors (mmlttb_minmaxlttb_host), blocking.  Pinned tensors
    are read in place by the kernels (the device buffer then holds no copy of the
    series, so the series may exceed device memory); pageable ones are staged."""
    _check_inputs(y, x, cuda=False)
    if y.is_cuda:
        raise ValueError("minmaxlttb_host takes host tensors")
    device = torch.device(device if device is not None else "cuda")
    n = y.numel()
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode)
    cap = max(min(n, n_out), 1)
    if out is None:
        out = torch.empty(cap, dtype=torch.int64)
    count = torch.zeros(1, dtype=torch.int64)
    inplace = y.is_pinned() and (x is None or x.is_pinned())
    need = host_buffer_bytes(yd, xk, n, n_out, r_ps, bm, inplace=inplace)
    if device_buffer is None:
        device_buffer = torch.empty(need, dtype=torch.uint8, device=device)
    if not device_buffer.is_cuda or out.is_cuda:
        raise ValueError("device_buffer must be a CUDA tensor and out a host tensor")
    _check(lib.mmlttb_minmaxlttb_host(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out, r_ps, bm,
        out.data_ptr(), out.numel(), count.data_ptr(), device_buffer.data_ptr(),
        device_buffer.numel(), _stream(device)), "mmlttb_minmaxlttb_host")
    return out[: int(count.item())]


def set_timing_events(start, stop):
    """Arm the one-shot events around the next streaming MinMax kernel
    (torch.cuda.Event(enable_timing=True) objects that have been recorded once, so
    that torch has created them; or None, None)."""
    _check(lib.mmlttb_set_timing_events(ctypes.c_void_p(start.cuda_event) if start is not None else None,
                                        ctypes.c_void_p(stop.cuda_event) if stop is not None else None),
           "mmlttb_set_timing_events")


def stream_variants():
    """[(unroll, min_blocks)] of the compiled stream-kernel variants."""
    out = []
    v = 0
    while True:
        u, b = _int(0), _int(0)
        if lib.mmlttb_stream_variant_info(v, ctypes.byref(u), ctypes.byref(b)) != OK:
            return out
        out.append((u.value, b.value))
        v += 1


def _tune_cache_path():
    return os.environ.get("MMLTTB_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mmlttb_tuning.json"))


def autotune(y, n_out=4000, r_ps=4, save=True):
    """Time every stream-kernel variant on MinMax preselection of y (a CUDA tensor),
    select the fastest for y's type on y's device, and record it in the tuning cache
    (JSON keyed by device name and y type).  Returns (variant, median ms)."""
    import json
    _check_inputs(y, None)
    yd = _ydt(y)
    n = y.numel()
    cap = min(n, (n_out * r_ps // 2) * 2 + 2)
    out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
    ws = torch.empty(workspace_bytes(OP_PRESELECT, yd, X_IMPLICIT, n, n_out, r_ps), dtype=torch.uint8,
                     device=y.device)
    v, ms = _int(0), ctypes.c_float(0.0)
    with torch.cuda.device(y.device):
        _check(lib.mmlttb_autotune(yd, y.data_ptr(), n, n_out, r_ps, out.data_ptr(), out.numel(),
                                   ws.data_ptr(), ws.numel(), _stream(y.device), ctypes.byref(v),
                                   ctypes.byref(ms)), "mmlttb_autotune")
    if save:
        path = _tune_cache_path()
        try:
            cache = json.load(open(path)) if os.path.exists(path) else {}
        except (OSError, ValueError):
            cache = {}
        cache[f"{torch.cuda.get_device_name(y.device)}/{'f32' if yd == F32 else 'f64'}"] = v.value
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return v.value, ms.value


class Tuning(ctypes.Structure):
    """mmlttb_tuning: stream-kernel variant, lanes-per-bin shift, k_tables rounds."""
    _fields_ = [("variant", _i32), ("group_shift", _i32), ("tab_rounds", _i32), ("reserved", _i32)]

    def as_dict(self):
        return {"variant": self.variant, "group_shift": self.group_shift, "tab_rounds": self.tab_rounds}


lib.mmlttb_stream_variant_threads.argtypes = [_int, ctypes.POINTER(_int)]
lib.mmlttb_set_tuning.argtypes = [_int, _int, _int, _i64, ctypes.POINTER(Tuning)]
lib.mmlttb_get_tuning.argtypes = [_int, _int, _int, _i64, ctypes.POINTER(Tuning)]
lib.mmlttb_autotune_tuple.argtypes = [_int, _vp, _int, _vp, _i64, _i64, _i32, _int, _vp, _i64, _vp, _sz, _vp,
                                      ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_float)]
lib.mmlttb_batch_tuning.argtypes = [_vp, ctypes.POINTER(Tuning)]
lib.mmlttb_batch_tuning_key.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int),
                                        ctypes.POINTER(_i64)]


def stream_variant_threads(variant):
    t = _int(0)
    _check(lib.mmlttb_stream_variant_threads(variant, ctypes.byref(t)), "mmlttb_stream_variant_threads")
    return t.value


def set_tuning(ydtype, xkind, binmode, n_in, variant, group_shift=0, tab_rounds=0):
    """Store a tuning for the key (current device, y type, x kind, bin mode, size class
    of n_in)."""
    t = Tuning(variant, group_shift, tab_rounds, 0)
    _check(lib.mmlttb_set_tuning(ydtype, xkind, binmode, n_in, ctypes.byref(t)), "mmlttb_set_tuning")


def get_tuning(ydtype, xkind, binmode, n_in):
    """The tuning calls with this key use (the stored one, else the default)."""
    t = Tuning()
    _check(lib.mmlttb_get_tuning(ydtype, xkind, binmode, n_in, ctypes.byref(t)), "mmlttb_get_tuning")
    return t.as_dict()


def clear_tunings():
    _check(lib.mmlttb_clear_tunings(), "mmlttb_clear_tunings")


def _size_class(n):
    c = 0
    while n >= 10 and c < 12:
        n //= 10
        c += 1
    return c


def autotune_tuple(y, n_out=4000, r_ps=4, x=None, binmode=BINS_INDEX, save=True):
    """Time every stream variant x lanes-per-bin shift on MinMax preselection of y (and
    x), then k_tables rounds on MinMaxLTTB of it; store the fastest tuning under the
    series' key and, with save, in the tuning cache (JSON keyed by device name, y type,
    x kind, bin mode and size class).  Returns (tuning dict, median stream ms)."""
    import json
    _check_inputs(y, x)
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode)
    n = y.numel()
    cap = max(1, min(n, (n_out * r_ps // 2) * 2 + 2))
    out = torch.empty(cap, dtype=torch.int64, device=y.device)
    wsb = max(workspace_bytes(OP_PRESELECT, yd, xk, n, n_out, r_ps, bm),
              workspace_bytes(OP_MINMAXLTTB, yd, xk, n, n_out, r_ps, bm))
    ws = torch.empty(wsb, dtype=torch.uint8, device=y.device)
    t, ms = Tuning(), ctypes.c_float(0.0)
    with torch.cuda.device(y.device):
        _check(lib.mmlttb_autotune_tuple(yd, y.data_ptr(), xk, x.data_ptr() if x is not None else None, n, n_out,
                                         r_ps, bm, out.data_ptr(), out.numel(), ws.data_ptr(), ws.numel(),
                                         _stream(y.device), ctypes.byref(t), ctypes.byref(ms)),
               "mmlttb_autotune_tuple")
    if save:
        path = _tune_cache_path()
        try:
            cache = json.load(open(path)) if os.path.exists(path) else {}
        except (OSError, ValueError):
            cache = {}
        key = f"{torch.cuda.get_device_name(y.device)}/tuple/{yd}/{xk}/{bm}/{_size_class(n)}"
        cache[key] = t.as_dict()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return t.as_dict(), ms.value


def autotune_batch(series, steps=10, warmup=3, shifts=(-1, 0, 1), rounds=(0, 2, 4, 7)):
    """Time the CUDA-graph replay of a batch of `series` (as for Batch) planned with
    every tuning tuple (stream variants x lanes-per-bin shifts x k_tables rounds), keep
    the fastest for the batch's tuning key, and return (tuning dict, median ms, all
    timings)."""
    b = Batch(series)
    key = b.tuning_key()
    b.close()
    timings = {}
    best, best_ms = None, float("inf")
    for v in range(len(stream_variants())):
        for g in shifts:
            for r in rounds:
                set_tuning(*key, v, g, r)
                b = Batch(series)
                for _ in range(warmup):
                    b.run(graph=True)
                ts = []
                for _ in range(steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    b.run(graph=True)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                b.close()
                ms = sorted(ts)[len(ts) // 2]
                timings[(v, g, r)] = ms
                if ms < best_ms:
                    best, best_ms = (v, g, r), ms
    set_tuning(*key, *best)
    return {"variant": best[0], "group_shift": best[1], "tab_rounds": best[2]}, best_ms, timings


def load_tuning(device=None):
    """Apply the cached tunings for `device` (if any were saved): stream variants per y
    type, and tuples per (y type, x kind, bin mode, size class)."""
    import json
    path = _tune_cache_path()
    if not os.path.exists(path):
        return {}
    cache = json.load(open(path))
    device = torch.device(device if device is not None else "cuda")
    name = torch.cuda.get_device_name(device)
    applied = {}
    with torch.cuda.device(device):
        for yd, key in ((F32, "f32"), (F64, "f64")):
            v = cache.get(f"{name}/{key}")
            if v is not None:
                _check(lib.mmlttb_set_stream_variant(yd, int(v)), "mmlttb_set_stream_variant")
                applied[key] = v
        for key, t in cache.items():
            parts = key.split("/")
            if len(parts) == 6 and parts[0] == name and parts[1] == "tuple":
                yd, xk, bm, c = (int(q) for q in parts[2:])
                set_tuning(yd, xk, bm, 10 ** c, t["variant"], t["group_shift"], t["tab_rounds"])
                applied[key] = t
    return applied


def set_stage_events(events):
    """Arm one-shot events between the kernels of the next call (recorded torch
    events: index 0 before the first kernel, k after the k-th)."""
    arr = (_vp * len(events))(*[e.cuda_event for e in events])
    _check(lib.mmlttb_set_stage_events(arr, len(events)), "mmlttb_set_stage_events")


def launch_count():
    """Kernels launched by the library from this thread so far."""
    return int(lib.mmlttb_launch_count())


# ---- line-chart rasterisation and visual metrics (include/mmlttb_raster.h) ----
_f64 = ctypes.c_double
lib.mmlttb_raster.argtypes = [_vp, _int, _vp, _int, _i64, _vp, _i64, _f64, _f64, _f64, _f64, _i32, _i32, _vp, _vp]
lib.mmlttb_raster_intensity.argtypes = [_vp, _i64, _vp, _vp]
lib.mmlttb_visual_counts.argtypes = [_vp, _vp, _i32, _i32, _i32, _vp, _vp]


def raster(y, extents, width, height, x=None, idx=None, mask=None):
    """Line chart of the points idx (all points when None) of series (x, y) on a
    width x height canvas (mmlttb_raster): per pixel the 16-bit mask of inked samples,
    OR-ed into `mask` (an int32 tensor of shape (height, width) holding the uint32 bit
    patterns; a zeroed one is made when None).  extents = (x0, x1, y0, y1)."""
    _check_inputs(y, x)
    if mask is None:
        mask = torch.zeros((height, width), dtype=torch.int32, device=y.device)
    elif mask.dtype != torch.int32 or tuple(mask.shape) != (height, width) or not mask.is_contiguous():
        raise ValueError("mask must be a contiguous int32 tensor of shape (height, width)")
    _on(mask, y.device, "mask")
    ip, k = None, 0
    if idx is not None:
        if idx.dtype != torch.int64 or idx.dim() != 1 or not idx.is_contiguous() or idx.device != y.device:
            raise ValueError("idx must be a contiguous 1-D int64 tensor on the device of y")
        ip, k = idx.data_ptr(), idx.numel()
    x0, x1, y0, y1 = (float(v) for v in extents)
    _check(lib.mmlttb_raster(y.data_ptr(), _ydt(y), x.data_ptr() if x is not None else None, _xkind(x),
                             y.numel(), ip, k, x0, x1, y0, y1, width, height, mask.data_ptr(),
                             _stream(y.device)), "mmlttb_raster")
    return mask


def intensity(mask):
    """8-bit intensities of a canvas of sample masks (mmlttb_raster_intensity)."""
    if mask.dtype != torch.int32 or not mask.is_contiguous() or not mask.is_cuda:
        raise ValueError("mask must be a contiguous int32 CUDA tensor")
    out = torch.empty(mask.shape, dtype=torch.uint8, device=mask.device)
    _check(lib.mmlttb_raster_intensity(mask.data_ptr(), mask.numel(), out.data_ptr(), _stream(mask.device)),
           "mmlttb_raster_intensity")
    return out


def visual_counts(ref, img, margin=20, sync=True):
    """(pixels differing by more than margin, sum of squared differences, conv-mask
    size) of two 8-bit images of the same shape (mmlttb_visual_counts); with
    sync=False the device int64[3] tensor."""
    if ref.dtype != torch.uint8 or img.dtype != torch.uint8 or ref.shape != img.shape or ref.dim() != 2:
        raise ValueError("ref and img must be uint8 images of the same (height, width)")
    if not (ref.is_contiguous() and img.is_contiguous()) or ref.device != img.device or not ref.is_cuda:
        raise ValueError("ref and img must be contiguous and on one CUDA device")
    counts = torch.empty(3, dtype=torch.int64, device=ref.device)
    h, w = ref.shape
    _check(lib.mmlttb_visual_counts(ref.data_ptr(), img.data_ptr(), w, h, margin, counts.data_ptr(),
                                    _stream(ref.device)), "mmlttb_visual_counts")
    if not sync:
        return counts
    return tuple(int(v) for v in counts.tolist())


def visual_metrics(ref, img, margin=20):
    """PEM_margin and MSE of img against the reference image ref, both over the
    conv-mask of ref (0 for an empty mask)."""
    over, sq, size = visual_counts(ref, img, margin)
    return {"pem": over / size if size else 0.0, "mse": sq / size if size else 0.0, "mask": size}


# ---- failure-detection diagnostics (include/mmlttb_diag.h) ----
DIAG_FUSED_BARRIER, DIAG_GRID_BARRIER, DIAG_MBARRIER = 0, 1, 2
lib.mmlttb_diag_wait_timeout.argtypes = [_int, _vp, _sz, _vp]


def diag_wait_timeout(which, workspace):
    """Run a bounded barrier wait that nothing satisfies (mmlttb_diag_wait_timeout);
    afterwards workspace_status(workspace) reports bit 1.  Asynchronous (about 2 s)."""
    if not workspace.is_cuda:
        raise ValueError("workspace must be a CUDA tensor")
    _check(lib.mmlttb_diag_wait_timeout(which, workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                        _stream(workspace.device)), "mmlttb_diag_wait_timeout")


CHECK_Y_NAN, CHECK_X_DECREASES, CHECK_X_NONFINITE = 0x1, 0x2, 0x4
lib.mmlttb_check_series.argtypes = [_vp, _int, _vp, _int, _i64, _vp, _vp]


def check_series(y, x=None):
    """The documented preconditions of a series checked on the device
    (mmlttb_check_series): a set of the violations found, of "y_nan",
    "x_decreases" and "x_nonfinite" (empty when none)."""
    _check_inputs(y, x)
    flags = torch.zeros(1, dtype=torch.int32, device=y.device)
    _check(lib.mmlttb_check_series(y.data_ptr(), _ydt(y), x.data_ptr() if x is not None else None, _xkind(x),
                                   y.numel(), flags.data_ptr(), _stream(y.device)), "mmlttb_check_series")
    f = int(flags.item())
    return {name for bit, name in ((CHECK_Y_NAN, "y_nan"), (CHECK_X_DECREASES, "x_decreases"),
                                   (CHECK_X_NONFINITE, "x_nonfinite")) if f & bit}


lib.mmlttb_set_single_path.argtypes = [_int]
lib.mmlttb_single_path.argtypes = [_int, _int, _int, _i64, _i64, _i32, _int]


def set_single_path(path):
    """Launch-path preference of this thread's single-series calls (PATH_AUTO,
    PATH_SPLIT, PATH_FUSED_TAIL or PATH_FUSED)."""
    _check(lib.mmlttb_set_single_path(path), "mmlttb_set_single_path")


lib.mmlttb_set_stream_staging.argtypes = [_int]
lib.mmlttb_get_stream_staging.argtypes = [ctypes.POINTER(_int)]


def set_stream_staging(enable):
    """Whether plans made from now on send small index bins of large launches to the
    staged (cp.async.bulk) MinMax stream (True) or to the register stream (False, the
    default)."""
    _check(lib.mmlttb_set_stream_staging(1 if enable else 0), "mmlttb_set_stream_staging")


def stream_staging():
    v = _int(0)
    _check(lib.mmlttb_get_stream_staging(ctypes.byref(v)), "mmlttb_get_stream_staging")
    return bool(v.value)


lib.mmlttb_stream_tiles.argtypes = [_int, _int, _int, _i64, _i64, _i32, _int, ctypes.POINTER(_i64)]


def stream_tiles(op, ydtype, xkind, n_in, n_out, r_ps=4, binmode=BINS_INDEX):
    """Bins per staged tile of a single-series call with these arguments here (0: the
    register stream)."""
    v = _i64(0)
    _check(lib.mmlttb_stream_tiles(op, ydtype, xkind, n_in, n_out, r_ps, binmode, ctypes.byref(v)),
           "mmlttb_stream_tiles")
    return int(v.value)


def single_path(op, ydtype, xkind, n_in, n_out, r_ps=4, binmode=BINS_INDEX):
    """The launch path a single-series call with these arguments takes here."""
    r = lib.mmlttb_single_path(op, ydtype, xkind, n_in, n_out, r_ps, binmode)
    _check(r if r < 0 else 0, "mmlttb_single_path")
    return r


class SeriesDesc(ctypes.Structure):
    """mmlttb_series_desc."""
    _fields_ = [("y", _vp), ("x", _vp), ("op", _i32), ("ydtype", _i32), ("xkind", _i32),
                ("binmode", _i32), ("r_ps", _i32), ("reserved", _i32), ("n_in", _i64),
                ("n_out", _i64), ("out_idx", _vp), ("out_cap", _i64), ("out_count", _vp)]


lib.mmlttb_batch_create.restype = _int
lib.mmlttb_batch_create.argtypes = [ctypes.POINTER(SeriesDesc), _i64, ctypes.POINTER(_vp)]
lib.mmlttb_batch_workspace_bytes.restype = _int
lib.mmlttb_batch_workspace_bytes.argtypes = [_vp, ctypes.POINTER(_sz)]
lib.mmlttb_batch_run.restype = _int
lib.mmlttb_batch_run.argtypes = [_vp, _vp, _sz, _vp]
lib.mmlttb_batch_run_graph.restype = _int
lib.mmlttb_batch_run_graph.argtypes = [_vp, _vp, _sz, _vp]
lib.mmlttb_batch_destroy.restype = _int
lib.mmlttb_batch_destroy.argtypes = [_vp]

_OPS = {"minmaxlttb": OP_MINMAXLTTB, "lttb": OP_LTTB, "preselect": OP_PRESELECT, "m4": OP_M4}


class Batch:
    """Many series in one launch sequence (mmlttb_batch_*).

    series: list of dicts with keys y (CUDA tensor), n_out, and optionally x, r_ps
    (default 4), op ("minmaxlttb" | "lttb" | "preselect"), binmode.  Outputs live in
    one int64 tensor; results() slices them after a sync."""

    def __init__(self, series, workspace=None):
        if not series:
            raise ValueError("empty batch")
        self.device = series[0]["y"].device
        self._keep = []
        caps = []
        descs = (SeriesDesc * len(series))()
        for i, s in enumerate(series):
            y, x = s["y"], s.get("x")
            _check_inputs(y, x)
            _on(y, self.device, "every series' y")
            op = _OPS[s.get("op", "minmaxlttb")]
            r_ps = int(s.get("r_ps", 4))
            n, n_out = y.numel(), int(s["n_out"])
            cap = (min(n, (n_out * r_ps // 2) * 2 + 2) if op == OP_PRESELECT
                   else min(n, 4 * (n_out // 4)) if op == OP_M4 else min(n, n_out))
            caps.append(max(cap, 0))
            d = descs[i]
            d.y = y.data_ptr()
            d.x = x.data_ptr() if x is not None else None
            d.op, d.ydtype, d.xkind = op, _ydt(y), _xkind(x)
            d.binmode, d.r_ps, d.reserved = _binmode(s.get("binmode", BINS_INDEX)), r_ps, 0
            d.n_in, d.n_out = n, n_out
            self._keep.append((y, x))
        offs = [0]
        for c in caps:
            offs.append(offs[-1] + c)
        self.offsets = offs
        self.out = torch.empty(max(offs[-1], 1), dtype=torch.int64, device=self.device)
        self.counts = torch.zeros(len(series), dtype=torch.int64, device=self.device)
        base, cbase = self.out.data_ptr(), self.counts.data_ptr()
        for i in range(len(series)):
            descs[i].out_idx = base + 8 * offs[i]
            descs[i].out_cap = caps[i]
            descs[i].out_count = cbase + 8 * i
        self._descs = descs
        h = _vp()
        _check(lib.mmlttb_batch_create(descs, len(series), ctypes.byref(h)), "mmlttb_batch_create")
        self._h = h
        b = ctypes.c_size_t(0)
        _check(lib.mmlttb_batch_workspace_bytes(h, ctypes.byref(b)), "mmlttb_batch_workspace_bytes")
        self.workspace_bytes = b.value
        self.workspace = _on(workspace, self.device, "workspace") if workspace is not None else torch.empty(
            self.workspace_bytes, dtype=torch.uint8, device=self.device)

    def run(self, graph=False):
        fn = lib.mmlttb_batch_run_graph if graph else lib.mmlttb_batch_run
        _check(fn(self._h, self.workspace.data_ptr(),
                  self.workspace.numel() * self.workspace.element_size(), _stream(self.device)),
               "mmlttb_batch_run_graph" if graph else "mmlttb_batch_run")

    def results(self):
        counts = self.counts.cpu().tolist()
        return [self.out[self.offsets[i]: self.offsets[i] + counts[i]] for i in range(len(counts))]

    def tuning(self):
        """The tuning the batch was planned with (mmlttb_batch_tuning)."""
        t = Tuning()
        _check(lib.mmlttb_batch_tuning(self._h, ctypes.byref(t)), "mmlttb_batch_tuning")
        return t.as_dict()

    def tuning_key(self):
        """(y type, x kind, bin mode, n_in) of the tuning key the batch was planned under."""
        a, b, c, n = _int(0), _int(0), _int(0), _i64(0)
        _check(lib.mmlttb_batch_tuning_key(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                           ctypes.byref(n)), "mmlttb_batch_tuning_key")
        return a.value, b.value, c.value, n.value

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize(self.device)
            lib.mmlttb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving
EBUSY = -10


class ServerConfig(ctypes.Structure):
    _fields_ = [("streams", _i32), ("reserved", _i32), ("max_batch", _i64), ("max_n_out", _i64),
                ("max_pending", _i64), ("workspace_bytes_per_stream", _i64)]


class Request(ctypes.Structure):
    _fields_ = [("series", _i64), ("start", _i64), ("end", _i64), ("n_out", _i64), ("r_ps", _i32),
                ("binmode", _i32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _i64), ("completed", _i64), ("rejected", _i64), ("batches", _i64),
                ("gpu_launches", _i64), ("mean_batch", ctypes.c_double), ("latency_p50_s", ctypes.c_double),
                ("latency_p99_s", ctypes.c_double), ("latency_max_s", ctypes.c_double),
                ("latency_mean_s", ctypes.c_double), ("overlapped_batches", _i64),
                ("max_batches_in_flight", _i64)]


lib.mmlttb_server_pool_bytes.restype = _int
lib.mmlttb_server_pool_bytes.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_sz)]
lib.mmlttb_server_create.restype = _int
lib.mmlttb_server_create.argtypes = [ctypes.POINTER(ServerConfig), _vp, _sz, ctypes.POINTER(_vp)]
lib.mmlttb_server_add_series.restype = _int
lib.mmlttb_server_add_series.argtypes = [_vp, _vp, _int, _vp, _int, _i64, ctypes.POINTER(_i64)]
lib.mmlttb_server_submit.restype = _int
lib.mmlttb_server_submit.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
lib.mmlttb_server_wait.restype = _int
lib.mmlttb_server_wait.argtypes = [_vp, ctypes.c_uint64, _vp, _i64, ctypes.POINTER(_i64),
                                   ctypes.POINTER(ctypes.c_double)]
lib.mmlttb_server_drain.restype = _int
lib.mmlttb_server_drain.argtypes = [_vp]
lib.mmlttb_server_replay.restype = _int
lib.mmlttb_server_replay.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double), _i64,
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_int)]
lib.mmlttb_server_get_stats.restype = _int
lib.mmlttb_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
lib.mmlttb_server_reset_stats.restype = _int
lib.mmlttb_server_reset_stats.argtypes = [_vp]
lib.mmlttb_server_destroy.restype = _int
lib.mmlttb_server_destroy.argtypes = [_vp]


class Server:
    """Zoom-window MinMaxLTTB server with continuous batching (mmlttb_server_*).

    Resident series are CUDA tensors the caller keeps alive; the device pool is a
    torch allocation owned by this object."""

    def __init__(self, streams=2, max_batch=256, max_n_out=4000, max_pending=1 << 20,
                 workspace_bytes_per_stream=256 << 20, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.cfg = ServerConfig(streams, 0, max_batch, max_n_out, max_pending, workspace_bytes_per_stream)
        nb = ctypes.c_size_t(0)
        _check(lib.mmlttb_server_pool_bytes(ctypes.byref(self.cfg), ctypes.byref(nb)), "mmlttb_server_pool_bytes")
        self.pool = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        h = _vp()
        with torch.cuda.device(self.device):
            _check(lib.mmlttb_server_create(ctypes.byref(self.cfg), self.pool.data_ptr(), nb.value,
                                            ctypes.byref(h)), "mmlttb_server_create")
        self._h = h
        self._series = []

    def add_series(self, y, x=None):
        _check_inputs(y, x)
        sid = _i64(0)
        _check(lib.mmlttb_server_add_series(self._h, y.data_ptr(), _ydt(y), x.data_ptr() if x is not None else None,
                                            _xkind(x), y.numel(), ctypes.byref(sid)), "mmlttb_server_add_series")
        self._series.append((y, x))
        return sid.value

    def submit(self, series, start, end, n_out, r_ps=4, binmode=BINS_INDEX):
        q = Request(series, start, end, n_out, r_ps, _binmode(binmode))
        rid = ctypes.c_uint64(0)
        rc = lib.mmlttb_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid))
        if rc != OK:
            raise MMLTTBError(rc, "mmlttb_server_submit")
        return rid.value

    def wait(self, rid):
        import numpy as np
        out = np.empty(self.cfg.max_n_out, dtype=np.int64)
        cnt = _i64(0)
        lat = ctypes.c_double(0.0)
        _check(lib.mmlttb_server_wait(self._h, rid, out.ctypes.data, out.size, ctypes.byref(cnt), ctypes.byref(lat)),
               "mmlttb_server_wait")
        return out[: cnt.value].copy(), lat.value

    def replay(self, requests, offsets_s):
        n = len(requests)
        arr = (Request * n)(*requests)
        offs = (ctypes.c_double * n)(*offsets_s)
        ids = (ctypes.c_uint64 * n)()
        st = (_int * n)()
        lib.mmlttb_server_replay(self._h, arr, offs, n, ids, st)
        return list(ids), list(st)

    def drain(self):
        _check(lib.mmlttb_server_drain(self._h), "mmlttb_server_drain")

    def stats(self):
        s = ServerStats()
        _check(lib.mmlttb_server_get_stats(self._h, ctypes.byref(s)), "mmlttb_server_get_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(lib.mmlttb_server_reset_stats(self._h), "mmlttb_server_reset_stats")

    def close(self):
        if getattr(self, "_h", None):
            lib.mmlttb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
