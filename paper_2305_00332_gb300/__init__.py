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
OP_PRESELECT, OP_LTTB, OP_MINMAXLTTB = 0, 1, 2

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
lib.mmlttb_workspace_status.restype = _int
lib.mmlttb_workspace_status.argtypes = [_vp, ctypes.POINTER(_int), _vp]
lib.mmlttb_host_buffer_bytes.restype = _int
lib.mmlttb_host_buffer_bytes.argtypes = [_int, _int, _i64, _i64, _i32, _int, ctypes.POINTER(_sz)]
lib.mmlttb_minmaxlttb_host.restype = _int
lib.mmlttb_minmaxlttb_host.argtypes = [_vp, _int, _vp, _int, _i64, _i64, _i32, _int, _vp, _i64, _vp,
                                       _vp, _sz, _vp]
lib.mmlttb_set_timing_events.restype = _int
lib.mmlttb_set_timing_events.argtypes = [_vp, _vp]
lib.mmlttb_launch_count.restype = ctypes.c_ulonglong


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


def _binmode(binmode):
    if binmode in (BINS_INDEX, "index"):
        return BINS_INDEX
    if binmode in (BINS_XWIDTH, "xwidth", "x"):
        return BINS_XWIDTH
    raise ValueError(f"unknown bin mode {binmode!r}")


def _check_inputs(y, x):
    if y.dim() != 1 or not y.is_contiguous():
        raise ValueError("y must be a contiguous 1-D tensor")
    if x is not None:
        if x.dim() != 1 or not x.is_contiguous() or x.numel() != y.numel():
            raise ValueError("x must be a contiguous 1-D tensor of the same length as y")
        if x.device != y.device:
            raise ValueError("x and y must be on the same device")


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
    return workspace  # the C ABI checks the size (MMLTTB_ENOSPC)


def _finish(out, count, sync):
    if not sync:
        return out, count
    return out[: int(count.item())]


def minmax_preselect(y, n_out, r_ps, x=None, binmode=BINS_INDEX, out=None, workspace=None, sync=True):
    """MinMax preselection (mmlttb_minmax_preselect): int64 indices of point 0, the
    per-bin argmin/argmax of floor(n_out*r_ps/2) bins, and point n-1."""
    _check_inputs(y, x)
    n = y.numel()
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode)
    cap = min(n, (n_out * r_ps // 2) * 2 + 2)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
    count = torch.empty(1, dtype=torch.int64, device=y.device)
    ws = _workspace(workspace_bytes(OP_PRESELECT, yd, xk, n, n_out, r_ps, bm), y.device, workspace)
    _check(lib.mmlttb_minmax_preselect(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out, r_ps, bm,
        out.data_ptr(), out.numel(), count.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), _stream(y.device)),
        "mmlttb_minmax_preselect")
    return _finish(out, count, sync)


def lttb(y, n_out, x=None, out=None, workspace=None, sync=True):
    """Plain LTTB on all points (mmlttb_lttb): min(n_out, n) int64 indices."""
    _check_inputs(y, x)
    n = y.numel()
    yd, xk = _ydt(y), _xkind(x)
    cap = min(n, n_out)
    if out is None:
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=y.device)
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
    count = torch.empty(1, dtype=torch.int64, device=y.device)
    ws = _workspace(workspace_bytes(OP_MINMAXLTTB, yd, xk, n, n_out, r_ps, bm), y.device, workspace)
    _check(lib.mmlttb_minmaxlttb(
        y.data_ptr(), yd, x.data_ptr() if x is not None else None, xk, n, n_out, r_ps, bm,
        out.data_ptr(), out.numel(), count.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), _stream(y.device)),
        "mmlttb_minmaxlttb")
    return _finish(out, count, sync)


def workspace_status(workspace):
    """Status word of a workspace after the calls that used it (blocking)."""
    st = ctypes.c_int(0)
    _check(lib.mmlttb_workspace_status(workspace.data_ptr(), ctypes.byref(st), _stream(workspace.device)),
           "mmlttb_workspace_status")
    return st.value


def host_buffer_bytes(ydtype, xkind, n_in, n_out, r_ps=4, binmode=BINS_INDEX):
    """Device bytes mmlttb_minmaxlttb_host needs (staged input, output, workspace)."""
    b = ctypes.c_size_t(0)
    _check(lib.mmlttb_host_buffer_bytes(ydtype, xkind, n_in, n_out, r_ps, _binmode(binmode),
                                        ctypes.byref(b)), "mmlttb_host_buffer_bytes")
    return b.value


def minmaxlttb_host(y, n_out, r_ps=4, x=None, binmode=BINS_INDEX, out=None, device_buffer=None,
                    device=None):
    """MinMaxLTTB on host tensors (mmlttb_minmaxlttb_host): copies in, runs, copies the
    indices back; blocking.  Pinned host tensors make the copies asynchronous DMA."""
    _check_inputs(y, x)
    if y.is_cuda:
        raise ValueError("minmaxlttb_host takes host tensors")
    device = torch.device(device if device is not None else "cuda")
    n = y.numel()
    yd, xk, bm = _ydt(y), _xkind(x), _binmode(binmode)
    cap = max(min(n, n_out), 1)
    if out is None:
        out = torch.empty(cap, dtype=torch.int64)
    count = torch.zeros(1, dtype=torch.int64)
    need = host_buffer_bytes(yd, xk, n, n_out, r_ps, bm)
    if device_buffer is None:
        device_buffer = torch.empty(need, dtype=torch.uint8, device=device)
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


def launch_count():
    """Kernels launched by the library from this thread so far."""
    return int(lib.mmlttb_launch_count())


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

_OPS = {"minmaxlttb": OP_MINMAXLTTB, "lttb": OP_LTTB, "preselect": OP_PRESELECT}


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
            op = _OPS[s.get("op", "minmaxlttb")]
            r_ps = int(s.get("r_ps", 4))
            n, n_out = y.numel(), int(s["n_out"])
            cap = min(n, (n_out * r_ps // 2) * 2 + 2) if op == OP_PRESELECT else min(n, n_out)
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
        self.workspace = workspace if workspace is not None else torch.empty(
            self.workspace_bytes, dtype=torch.uint8, device=self.device)

    def run(self, graph=False):
        fn = lib.mmlttb_batch_run_graph if graph else lib.mmlttb_batch_run
        _check(fn(self._h, self.workspace.data_ptr(),
                  self.workspace.numel() * self.workspace.element_size(), _stream(self.device)),
               "mmlttb_batch_run_graph" if graph else "mmlttb_batch_run")

    def results(self):
        counts = self.counts.cpu().tolist()
        return [self.out[self.offsets[i]: self.offsets[i] + counts[i]] for i in range(len(counts))]

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
