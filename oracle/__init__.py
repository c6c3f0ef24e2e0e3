"""ctypes loader of the MinMaxLTTB oracle -- TEST INFRASTRUCTURE ONLY.

The oracle (mmlttb_oracle.c) is a plain single-threaded CPU statement of the
method of arXiv 2305.00332 (MinMax preselection, Sec. 3; LTTB, Sec. 2.2.1).  Only
the tests, the package smoke check and the benchmark's CPU-baseline leg may use
it; the product path never imports this package.  Inputs are numpy arrays on the
host; results are numpy int64 index arrays.
"""
import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_DIR, "mmlttb_oracle.c")
LIB = os.path.join(_DIR, "liboracle.so")

# -ffp-contract=off: every product and sum is rounded on its own (no FMA), also on
# aarch64 where GCC contracts by default.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]

F32, F64 = 0, 1
X_IMPLICIT, X_I64, X_F64 = 0, 1, 2
BINS_INDEX, BINS_XWIDTH = 0, 1
NAN_AWARE = 0x10


def compile_oracle(src=SRC, out=LIB, extra=()):
    """Compile an oracle source into a shared library (gcc)."""
    cmd = ["gcc", *CFLAGS, *extra, src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _fresh():
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC)


def load(path=None):
    """Load (building first when stale) an oracle shared library."""
    if path is None:
        if not _fresh():
            compile_oracle()
        path = LIB
    lib = ctypes.CDLL(path)
    i64, i32, vp, cint = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int
    lib.mmo_minmax_bins.restype = i64
    lib.mmo_minmax_bins.argtypes = [vp, cint, vp, cint, i64, i64, cint, vp, vp]
    lib.mmo_minmax_preselect.restype = i64
    lib.mmo_minmax_preselect.argtypes = [vp, cint, vp, cint, i64, i64, i32, cint, vp]
    lib.mmo_lttb_positions.restype = i64
    lib.mmo_lttb_positions.argtypes = [vp, cint, vp, cint, vp, i64, i64, vp]
    lib.mmo_lttb.restype = i64
    lib.mmo_lttb.argtypes = [vp, cint, vp, cint, i64, i64, vp]
    lib.mmo_m4.restype = i64
    lib.mmo_m4.argtypes = [vp, cint, vp, cint, i64, i64, cint, vp]
    lib.mmo_minmaxlttb.restype = i64
    lib.mmo_minmaxlttb.argtypes = [vp, cint, vp, cint, i64, i64, i32, cint, vp]
    dbl = ctypes.c_double
    lib.mmo_raster.restype = i64
    lib.mmo_raster.argtypes = [vp, cint, vp, cint, i64, vp, i64, dbl, dbl, dbl, dbl, cint, cint, vp]
    lib.mmo_raster_intensity.restype = None
    lib.mmo_raster_intensity.argtypes = [vp, i64, vp]
    lib.mmo_visual_counts.restype = None
    lib.mmo_visual_counts.argtypes = [vp, vp, cint, cint, cint, vp]
    return lib


class Oracle:
    """numpy front end of one oracle library build."""

    def __init__(self, path=None):
        self.lib = load(path)

    @staticmethod
    def _y(y):
        y = np.ascontiguousarray(y)
        if y.dtype == np.float32:
            return y, F32
        if y.dtype == np.float64:
            return y, F64
        raise TypeError(f"y dtype {y.dtype}")

    @staticmethod
    def _x(x, n):
        if x is None:
            return None, X_IMPLICIT, None
        x = np.ascontiguousarray(x)
        if len(x) != n:
            raise ValueError("x and y lengths differ")
        if x.dtype == np.int64:
            return x, X_I64, x.ctypes.data
        if x.dtype == np.float64:
            return x, X_F64, x.ctypes.data
        raise TypeError(f"x dtype {x.dtype}")

    @staticmethod
    def _bm(binmode, nan_aware=False):
        bm = {"index": BINS_INDEX, "xwidth": BINS_XWIDTH, BINS_INDEX: BINS_INDEX,
              BINS_XWIDTH: BINS_XWIDTH}[binmode]
        return bm | (NAN_AWARE if nan_aware else 0)

    @staticmethod
    def _rc(r, what):
        if r < 0:
            raise ValueError(f"oracle {what} returned {r}")
        return r

    def minmax_bins(self, y, B, x=None, binmode="index", nan_aware=False):
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        imin = np.empty(B, np.int64)
        imax = np.empty(B, np.int64)
        self._rc(self.lib.mmo_minmax_bins(y.ctypes.data, yd, xp, xk, len(y), B, self._bm(binmode, nan_aware),
                                          imin.ctypes.data, imax.ctypes.data), "minmax_bins")
        return imin, imax

    def minmax_preselect(self, y, n_out, r_ps, x=None, binmode="index", nan_aware=False):
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        B = max(n_out * r_ps // 2, 1)
        out = np.empty(2 * B + 2, np.int64)
        m = self._rc(self.lib.mmo_minmax_preselect(y.ctypes.data, yd, xp, xk, len(y), n_out, r_ps,
                                                   self._bm(binmode, nan_aware), out.ctypes.data), "preselect")
        return out[:m].copy()

    def lttb(self, y, n_out, x=None):
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        out = np.empty(max(min(n_out, len(y)), 1), np.int64)
        m = self._rc(self.lib.mmo_lttb(y.ctypes.data, yd, xp, xk, len(y), n_out, out.ctypes.data),
                     "lttb")
        return out[:m].copy()

    def lttb_positions(self, y, idx, n_out, x=None):
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(max(min(n_out, len(idx)), 1), np.int64)
        m = self._rc(self.lib.mmo_lttb_positions(y.ctypes.data, yd, xp, xk, idx.ctypes.data, len(idx),
                                                 n_out, out.ctypes.data), "lttb_positions")
        return out[:m].copy()

    def m4(self, y, n_out, x=None, binmode="index", nan_aware=False):
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        out = np.empty(max(4 * (n_out // 4), 1), np.int64)
        m = self._rc(self.lib.mmo_m4(y.ctypes.data, yd, xp, xk, len(y), n_out, self._bm(binmode, nan_aware),
                                     out.ctypes.data), "m4")
        return out[:m].copy()

    def minmaxlttb(self, y, n_out, r_ps=4, x=None, binmode="index"):
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        out = np.empty(max(min(n_out, len(y)), 1), np.int64)
        m = self._rc(self.lib.mmo_minmaxlttb(y.ctypes.data, yd, xp, xk, len(y), n_out, r_ps,
                                             self._bm(binmode), out.ctypes.data), "minmaxlttb")
        return out[:m].copy()


    def raster(self, y, extents, width, height, x=None, idx=None, mask=None):
        """Sample masks (uint32, height x width) of the line chart through points idx
        (all points when None), R19; extents = (x0, x1, y0, y1)."""
        y, yd = self._y(y)
        x, xk, xp = self._x(x, len(y))
        if mask is None:
            mask = np.zeros((height, width), np.uint32)
        ip, k = None, 0
        if idx is not None:
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            ip, k = idx.ctypes.data, len(idx)
        x0, x1, y0, y1 = (float(v) for v in extents)
        self._rc(self.lib.mmo_raster(y.ctypes.data, yd, xp, xk, len(y), ip, k, x0, x1, y0, y1,
                                     width, height, mask.ctypes.data), "raster")
        return mask

    def intensity(self, mask):
        mask = np.ascontiguousarray(mask, dtype=np.uint32)
        out = np.empty(mask.shape, np.uint8)
        self.lib.mmo_raster_intensity(mask.ctypes.data, mask.size, out.ctypes.data)
        return out

    def visual_counts(self, ref, img, margin=20):
        """(pixels differing by more than margin, sum of squared differences, mask size)."""
        ref = np.ascontiguousarray(ref, dtype=np.uint8)
        img = np.ascontiguousarray(img, dtype=np.uint8)
        counts = np.zeros(3, np.int64)
        h, w = ref.shape
        self.lib.mmo_visual_counts(ref.ctypes.data, img.ctypes.data, w, h, margin, counts.ctypes.data)
        return tuple(int(v) for v in counts)


_default = None


def oracle():
    """The shared default oracle instance (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
