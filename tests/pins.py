"""Pins of the oracle: checks against things other than the oracle itself.

Each check takes an oracle front end (oracle.Oracle) and raises AssertionError on a
mismatch.  What pins what:
  - worked examples: hand-derived cases in tests/golden/worked_examples.json;
  - MinMax: numpy.argmin / numpy.argmax (first occurrence) on every bin, bins
    built by point membership (a different statement of the bin layout);
  - x-width bins: brute-force membership (largest i with e_i <= x_p) in Python
    integers;
  - LTTB: exact rational arithmetic (fractions.Fraction) with the textbook
    shoelace area, on inputs where FP64 is provably exact (small integers,
    power-of-two bucket sizes), so the choice must match bit for bit;
  - general inputs: the chosen point's exact area is the bucket's exact maximum
    up to FP64 rounding;
  - invariants and symmetries that hold for any input.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_examples.json")


def rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- references
def bin_members_index(n, B):
    """Interior point p (1..n-2) lies in bin ceil(p*B/(n-2)) - 1 (equal-count bins)."""
    N = n - 2
    bins = [[] for _ in range(B)]
    for p in range(1, n - 1):
        bins[-(-p * B // N) - 1].append(p)
    return bins


def bin_members_xwidth(x, B):
    """Interior point p lies in the largest bin i with x0 + floor(i*D/B) <= x_p."""
    n = len(x)
    x = [int(v) for v in x]
    x0, D = x[0], x[-1] - x[0]
    edges = [x0 + (i * D) // B for i in range(B)]
    bins = [[] for _ in range(B)]
    for p in range(1, n - 1):
        i = max(k for k in range(B) if edges[k] <= x[p])
        bins[i].append(p)
    return bins


def bin_members_xwidth_f64(x, B, interior=True):
    """float64 x (R17): e_i = x0 + (i*D)/B with every operation rounded as IEEE
    doubles (Python floats), point p in the largest bin i with e_i <= x_p."""
    x = [float(v) for v in x]
    x0, D = x[0], x[-1] - x[0]
    edges = [x0 + (float(i) * D) / float(B) for i in range(B)]
    bins = [[] for _ in range(B)]
    pts = range(1, len(x) - 1) if interior else range(len(x))
    for p in pts:
        bins[max(k for k in range(B) if edges[k] <= x[p])].append(p)
    return bins


def minmax_reference(y, bins):
    """Per bin (argmin, argmax) by numpy (first occurrence), -1 for empty bins."""
    out = []
    for members in bins:
        if not members:
            out.append((-1, -1))
            continue
        a, b = members[0], members[-1] + 1
        seg = np.asarray(y[a:b])
        out.append((a + int(np.argmin(seg)), a + int(np.argmax(seg))))
    return out


def preselect_reference(y, bins):
    n = len(y)
    if n == 0:
        return []
    if n == 1:
        return [0]
    sel = [0]
    for lo, hi in minmax_reference(y, bins):
        if lo < 0:
            continue
        sel.extend(sorted({lo, hi}))
    sel.append(n - 1)
    return sel


def lttb_exact(X, Y, idx, n_out):
    """LTTB in exact rational arithmetic.  Position p (1..m-2) lies in bucket
    ceil(p*K/(m-2)) - 1; twice the triangle area is the shoelace sum
    |xa(yb-yc) + xb(yc-ya) + xc(ya-yb)|; ties go to the lowest position."""
    m = len(idx)
    if n_out >= m:
        return list(idx)
    K, N = n_out - 2, m - 2
    buckets = [[] for _ in range(K)]
    for p in range(1, m - 1):
        buckets[-(-p * K // N) - 1].append(p)
    out = [idx[0]]
    a = 0
    for j in range(K):
        nxt = buckets[j + 1] if j + 1 < K else [m - 1]
        xc = Fraction(sum(Fraction(X[idx[p]]) for p in nxt), len(nxt))
        yc = Fraction(sum(Fraction(Y[idx[p]]) for p in nxt), len(nxt))
        xa, ya = Fraction(X[idx[a]]), Fraction(Y[idx[a]])
        best, pick = None, None
        for p in buckets[j]:
            xb, yb = Fraction(X[idx[p]]), Fraction(Y[idx[p]])
            area = abs(xa * (yb - yc) + xb * (yc - ya) + xc * (ya - yb))
            if best is None or area > best:
                best, pick = area, p
        out.append(idx[pick])
        a = pick
    out.append(idx[m - 1])
    return out


def lttb_buckets(m, n_out):
    K, N = n_out - 2, m - 2
    buckets = [[] for _ in range(K)]
    for p in range(1, m - 1):
        buckets[-(-p * K // N) - 1].append(p)
    return buckets


# ---------------------------------------------------------------- checks
def check_worked_examples(o):
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        if "y_hex" in c:  # exact float64 inputs (cases G and H depend on every bit)
            y = np.array([float.fromhex(h) for h in c["y_hex"]], np.float64)
        else:
            y = np.array(c["y"], np.float64)
        x = np.array(c["x"], np.int64) if c["x"] is not None else None
        if c["op"] == "lttb":
            got = o.lttb(y, c["n_out"], x=x)
        elif c["op"] == "preselect":
            got = o.minmax_preselect(y, c["n_out"], c["r_ps"], x=x, binmode=c["binmode"])
        else:
            got = o.minmaxlttb(y, c["n_out"], c["r_ps"], x=x, binmode=c["binmode"])
        assert list(got) == c["expect"], (c["name"], list(got), c["expect"])
        if "preselected" in c:
            pre = o.minmax_preselect(y, c["n_out"], c["r_ps"], x=x, binmode=c["binmode"])
            assert list(pre) == c["preselected"], (c["name"], list(pre))
        if "expect_lttb" in c:
            assert list(o.lttb(y, c["n_out"], x=x)) == c["expect_lttb"], c["name"]


def _series_zoo(seed, n):
    r = rng(seed)
    yield np.cumsum(r.standard_normal(n)).astype(np.float32)
    yield np.cumsum(r.standard_normal(n)).astype(np.float64)
    yield r.integers(-3, 4, n).astype(np.float32)              # many ties
    yield np.array([-0.0, 0.0, -1.0, 1.0])[r.integers(0, 4, n)].astype(np.float64)  # signed zeros
    yield np.full(n, 2.5, np.float32)                           # constant


def check_minmax_index_bins(o):
    for seed in range(6):
        r = rng(100 + seed)
        for n in (3, 4, 5, 17, 64, 301):
            for y in _series_zoo(seed * 1000 + n, n):
                for B in sorted({1, 2, 3, max(1, (n - 2) // 3), max(1, n - 2), n + 3, int(r.integers(1, n + 5))}):
                    imin, imax = o.minmax_bins(y, B)
                    ref = minmax_reference(y, bin_members_index(n, B))
                    assert list(zip(imin.tolist(), imax.tolist())) == ref, (n, B, y.dtype)


def _increasing_x(r, n, repeats):
    gaps = r.integers(0 if repeats else 1, 6, n)
    gaps[0] = 0
    if n > 4:
        gaps[r.integers(1, n)] += 40  # a big gap: empty bins
    return (np.cumsum(gaps) - 7).astype(np.int64)


def check_minmax_xwidth_bins(o):
    for seed in range(8):
        r = rng(200 + seed)
        for n in (3, 5, 12, 50, 123):
            x = _increasing_x(r, n, repeats=seed % 2 == 1)
            for y in _series_zoo(seed * 77 + n, n):
                for B in (1, 2, 3, 7, max(1, n // 2), n + 2):
                    imin, imax = o.minmax_bins(y, B, x=x, binmode="xwidth")
                    ref = minmax_reference(y, bin_members_xwidth(x, B))
                    assert list(zip(imin.tolist(), imax.tolist())) == ref, (n, B, seed)


def check_minmax_xwidth_f64(o):
    """float64 x with fractional, uneven spacing, repeated values and big gaps."""
    for seed in range(6):
        r = rng(900 + seed)
        for n in (3, 7, 50, 321):
            g = r.exponential(0.7, n)
            g[0] = 0.0
            if seed % 2:
                g[r.integers(1, n, max(1, n // 5))] = 0.0  # repeated x
            if n > 4:
                g[r.integers(1, n)] += 50.0
            x = np.cumsum(g) - 3.3
            for y in _series_zoo(seed * 13 + n, n):
                for B in (1, 2, 5, 17, n + 1):
                    imin, imax = o.minmax_bins(y, B, x=x, binmode="xwidth")
                    ref = minmax_reference(y, bin_members_xwidth_f64(x, B))
                    assert list(zip(imin.tolist(), imax.tolist())) == ref, (n, B, seed)
                for n_out in (4, 12):
                    got = o.m4(y, n_out, x=x, binmode="xwidth")
                    assert list(got) == m4_reference(y, bin_members_xwidth_f64(x, n_out // 4, interior=False))
        # integer-valued float64 x on a grid: edges fall exactly on points
        for n in (9, 41, 200):
            x = np.arange(n, dtype=np.float64) * 2.0 + 1.0
            y = np.cumsum(r.standard_normal(n))
            for B in (2, 4, n - 1, (n - 1) // 2):
                imin, imax = o.minmax_bins(y, B, x=x, binmode="xwidth")
                assert list(zip(imin.tolist(), imax.tolist())) == minmax_reference(y, bin_members_xwidth_f64(x, B)), (n, B)


def _nan_series(r, n, dtype):
    y = np.cumsum(r.standard_normal(n)).astype(dtype)
    if n:
        y[r.integers(0, n, max(1, n // 9))] = np.nan
    return y


def check_nan_aware(o):
    """NaN-aware MinMax and M4 against numpy argmin/argmax, which return a bin's
    first NaN when it holds one (R18)."""
    for seed in range(5):
        r = rng(950 + seed)
        for n in (3, 10, 77, 400):
            for dt in (np.float32, np.float64):
                y = _nan_series(r, n, dt)
                for B in (1, 3, 10, n + 2):
                    imin, imax = o.minmax_bins(y, B, nan_aware=True)
                    ref = minmax_reference(y, bin_members_index(n, B))
                    assert list(zip(imin.tolist(), imax.tolist())) == ref, (n, B, seed)
                for n_out, r_ps in ((3, 2), (10, 4)):
                    got = o.minmax_preselect(y, n_out, r_ps, nan_aware=True)
                    assert list(got) == preselect_reference(y, bin_members_index(n, n_out * r_ps // 2))
                for n_out in (4, 16, 40):
                    got = o.m4(y, n_out, nan_aware=True)
                    assert list(got) == m4_reference(y, m4_members_index(n, n_out // 4))
                x = _increasing_x(r, n, repeats=True)
                got = o.minmax_preselect(y, 5, 4, x=x, binmode="xwidth", nan_aware=True)
                assert list(got) == preselect_reference(y, bin_members_xwidth(x, 10))


def check_preselect(o):
    for seed in range(5):
        r = rng(300 + seed)
        for n in (0, 1, 2, 3, 9, 40, 257):
            for y in _series_zoo(seed + n, n):
                for n_out, r_ps in ((1, 2), (3, 2), (5, 4), (10, 3), (7, 1)):
                    B = n_out * r_ps // 2
                    got = o.minmax_preselect(y, n_out, r_ps)
                    ref = preselect_reference(y, bin_members_index(n, B)) if n >= 2 else list(range(n))
                    assert list(got) == ref, (n, n_out, r_ps)
            if n >= 3:
                x = _increasing_x(r, n, repeats=True)
                y = np.cumsum(r.standard_normal(n))
                got = o.minmax_preselect(y, 6, 4, x=x, binmode="xwidth")
                assert list(got) == preselect_reference(y, bin_members_xwidth(x, 12))


def _exact_case(r, K, s, n_extra=0):
    """m = K*s + 2 positions, every bucket of size s (a power of two)."""
    m = K * s + 2
    n = m + n_extra
    y = r.integers(-20, 21, n).astype(np.float64)
    idx = np.sort(r.choice(n, size=m, replace=False)) if n_extra else np.arange(n)
    return y, idx


def check_lttb_exact(o):
    for seed in range(40):
        r = rng(400 + seed)
        K = int(r.integers(1, 12))
        s = int(r.choice([1, 2, 4, 8]))
        # all points
        y, idx = _exact_case(r, K, s)
        X = np.arange(len(y))
        ref = lttb_exact(X, y, list(range(len(y))), K + 2)
        assert list(o.lttb(y, K + 2)) == ref, ("lttb", seed)
        assert list(o.lttb(y.astype(np.float32), K + 2)) == ref, ("lttb f32", seed)
        # explicit int64 x with small gaps
        xg = np.cumsum(r.integers(1, 4, len(y))).astype(np.int64)
        ref = lttb_exact(xg, y, list(range(len(y))), K + 2)
        assert list(o.lttb(y, K + 2, x=xg)) == ref, ("lttb x", seed)
        # a subset of positions (the path LTTB takes after preselection)
        y, idx = _exact_case(r, K, s, n_extra=int(r.integers(1, 30)))
        X = np.arange(len(y))
        ref = lttb_exact(X, y, list(idx), K + 2)
        assert list(o.lttb_positions(y, idx, K + 2)) == ref, ("positions", seed)


def check_lttb_general(o):
    """Random floats: each pick attains the exact maximum area of its bucket
    (given the previous pick) up to a relative 1e-9."""
    for seed in range(6):
        r = rng(500 + seed)
        n = int(r.integers(20, 200))
        n_out = int(r.integers(3, max(4, n // 3)))
        y = np.cumsum(r.standard_normal(n))
        out = o.lttb(y, n_out)
        m, K = n, n_out - 2
        buckets = lttb_buckets(m, n_out)
        for j in range(K):
            a, pick = int(out[j]), int(out[j + 1])
            assert pick in buckets[j]
            nxt = buckets[j + 1] if j + 1 < K else [m - 1]
            xc = Fraction(sum(int(p) for p in nxt), len(nxt))
            yc = sum(Fraction(float(y[p])) for p in nxt) / len(nxt)
            xa, ya = Fraction(a), Fraction(float(y[a]))
            area = lambda p: abs(xa * (Fraction(float(y[p])) - yc) + p * (yc - ya) + xc * (ya - Fraction(float(y[p]))))
            best = max(area(p) for p in buckets[j])
            assert area(pick) >= best * (1 - Fraction(1, 10**9)), (seed, j)


def check_invariants(o):
    for seed in range(6):
        r = rng(600 + seed)
        n = int(r.integers(50, 3000))
        y = np.cumsum(r.standard_normal(n)).astype(np.float32 if seed % 2 else np.float64)
        for n_out in (3, 4, 17, max(3, n // 10), n - 1, n, n + 5):
            for r_ps in (2, 3, 4, 8):
                out = o.minmaxlttb(y, n_out, r_ps)
                lt = o.lttb(y, n_out)
                if n_out >= n:
                    assert list(out) == list(range(n)) and list(lt) == list(range(n))
                    continue
                for res in (out, lt):
                    assert len(res) == n_out
                    assert res[0] == 0 and res[-1] == n - 1
                    assert np.all(np.diff(res) > 0)
                # one pick per LTTB bucket (plain LTTB over all points)
                for j, b in enumerate(lttb_buckets(n, n_out)):
                    assert lt[j + 1] in b
                if r_ps * n_out >= n:
                    assert list(out) == list(lt)
                else:
                    pre = o.minmax_preselect(y, n_out, r_ps)
                    assert set(out.tolist()) <= set(pre.tolist())
                    pos = {v: i for i, v in enumerate(pre.tolist())}
                    for j, b in enumerate(lttb_buckets(len(pre), n_out)):
                        assert pos[int(out[j + 1])] in b
        # x-width bins: uneven bins can hold many points, so the r_ps*n_out >= n
        # branch (plain LTTB on all points, R15) differs from preselecting first
        x = _increasing_x(r, n, repeats=False)
        for n_out in (max(3, n // 3), max(3, n // 2)):
            for r_ps in (2, 4):
                got = o.minmaxlttb(y, n_out, r_ps, x=x, binmode="xwidth")
                if r_ps * n_out >= n:
                    assert list(got) == list(o.lttb(y, n_out, x=x))
                else:
                    pre = o.minmax_preselect(y, n_out, r_ps, x=x, binmode="xwidth")
                    assert set(got.tolist()) <= set(pre.tolist())


def check_symmetries(o):
    for seed in range(6):
        r = rng(700 + seed)
        n = int(r.integers(30, 600))
        y = np.cumsum(r.standard_normal(n)) if seed % 2 else r.integers(-50, 51, n).astype(np.float64)
        n_out = int(r.integers(3, n // 4))
        x2 = (2 * np.arange(n)).astype(np.int64)
        for r_ps in (2, 4):
            base = o.minmaxlttb(y, n_out, r_ps)
            # y -> -y negates every FP64 sum, mean and area term exactly and swaps
            # argmin/argmax per bin: the selection is unchanged
            assert list(o.minmaxlttb(-y, n_out, r_ps)) == list(base)
            # x = 2*index scales every x difference, product and mean exactly by 2
            assert list(o.minmaxlttb(y, n_out, r_ps, x=x2)) == list(base)
        assert list(o.lttb(-y, n_out)) == list(o.lttb(y, n_out))
        # shift by an integer on exact data (small integers, power-of-two buckets)
        K, s = int(r.integers(1, 10)), int(r.choice([1, 2, 4]))
        ye = r.integers(-50, 51, K * s + 2).astype(np.float64)
        assert list(o.lttb(ye + 1000.0, K + 2)) == list(o.lttb(ye, K + 2))


def check_constant_series(o):
    for n in (5, 37, 200):
        y = np.full(n, 3.0, np.float32)
        for n_out in (3, 5, 11):
            if n_out >= n:
                continue
            expect = [0] + [b[0] for b in lttb_buckets(n, n_out)] + [n - 1]
            assert list(o.lttb(y, n_out)) == expect
        pre = o.minmax_preselect(y, 4, 2)
        B = 4
        expect = [0] + [b[0] for b in bin_members_index(n, B) if b] + [n - 1]
        assert list(pre) == expect


def m4_members_index(n, B):
    """Point p (0..n-1) lies in bin ceil((p+1)*B/n) - 1: the bins [floor(i n/B), floor((i+1) n/B))."""
    bins = [[] for _ in range(B)]
    for p in range(n):
        bins[-(-(p + 1) * B // n) - 1].append(p)
    return bins


def m4_members_xwidth(x, B):
    """Point p lies in the largest bin i with x0 + floor(i*D/B) <= x_p (all points)."""
    x = [int(v) for v in x]
    x0, D = x[0], x[-1] - x[0]
    edges = [x0 + (i * D) // B for i in range(B)]
    bins = [[] for _ in range(B)]
    for p in range(len(x)):
        bins[max(k for k in range(B) if edges[k] <= x[p])].append(p)
    return bins


def m4_reference(y, bins):
    out = []
    for members in bins:
        if not members:
            continue
        a, b = members[0], members[-1] + 1
        seg = np.asarray(y[a:b])
        out.extend(sorted({a, a + int(np.argmin(seg)), a + int(np.argmax(seg)), b - 1}))
    return out


def check_m4(o):
    """M4 against numpy argmin/argmax plus the bins' first and last members."""
    for seed in range(5):
        r = rng(800 + seed)
        for n in (1, 2, 3, 7, 40, 333):
            for y in _series_zoo(seed * 31 + n, n):
                for n_out in (4, 5, 8, 12, 4 * n + 4, 101):
                    B = n_out // 4
                    assert list(o.m4(y, n_out)) == m4_reference(y, m4_members_index(n, B)), (n, n_out)
                if n >= 2:
                    x = _increasing_x(r, n, repeats=seed % 2 == 1)
                    for n_out in (4, 12, 40):
                        got = o.m4(y, n_out, x=x, binmode="xwidth")
                        assert list(got) == m4_reference(y, m4_members_xwidth(x, n_out // 4)), (n, n_out)


# ---- line-chart rasterisation and visual metrics (R19-R21) ----------------------

def _sample_points(c, r):
    """The 16 sample points of pixel (c, r) as exact fractions, bit index k*4 + i."""
    from fractions import Fraction as F
    return [(k * 4 + i, F(c) + F(2 * i + 1, 8), F(r) + F(2 * k + 1, 8)) for k in range(4) for i in range(4)]


def _exact_inked(sx, sy, ax, ay, bx, by):
    """Exact squared distance from a sample to a segment (all Fractions)."""
    dx, dy = bx - ax, by - ay
    l2 = dx * dx + dy * dy
    t = 0
    if l2 > 0:
        t = ((sx - ax) * dx + (sy - ay) * dy) / l2
        t = min(max(t, 0), 1)
    ex, ey = sx - (ax + t * dx), sy - (ay + t * dy)
    return ex * ex + ey * ey


def check_raster_closed_forms(o):
    """A horizontal line through the centre of row r inks all 16 samples of row r and
    8 of rows r-1 and r+1 (sample offsets 1/8, 3/8, 5/8, 7/8 at distances up to 1);
    a vertical line likewise for columns; intensity (16ths*255+8)/16."""
    W, H = 10, 7
    for r in range(1, H - 1):
        yv = H - (r + 0.5)  # py = (y1 - y) * H/(y1 - y0) with extents (0, W, 0, H)
        img = o.intensity(o.raster(np.array([yv, yv]), (0, W, 0, H), W, H, x=np.array([0.0, float(W)])))
        want = np.zeros((H, W), np.uint8)
        want[r, :] = 255
        want[r - 1, :] = 128
        want[r + 1, :] = 128
        assert np.array_equal(img, want), (r, img)
    for c in range(1, W - 1):
        xv = c + 0.5
        img = o.intensity(o.raster(np.array([0.0, float(H)]), (0, W, 0, H), W, H, x=np.array([xv, xv])))
        want = np.zeros((H, W), np.uint8)
        want[:, c] = 255
        want[:, c - 1] = 128
        want[:, c + 1] = 128
        assert np.array_equal(img, want), (c, img)
    # a sample at distance exactly 1 is inked: a line at py = 3.125 reaches the
    # samples at sy = 2.125 (row 2 fully inked) and sy = 4.125 (4 samples of row 4)
    img = o.intensity(o.raster(np.array([H - 3.125] * 2), (0, W, 0, H), W, H, x=np.array([0.0, float(W)])))
    want = np.zeros((H, W), np.uint8)
    want[2:4, :] = 255
    want[4, :] = (4 * 255 + 8) // 16
    assert np.array_equal(img, want), img
    # intensity rounding
    for inked in range(17):
        m = np.array([[(1 << inked) - 1]], np.uint32)
        assert int(o.intensity(m)[0, 0]) == (inked * 255 + 8) // 16


def check_raster_brute_force(o):
    """Random short segments with endpoints on a 1/8 grid: every pixel's sample mask
    equals the exact-arithmetic test (samples within 1e-6 of the boundary excepted,
    where float rounding may decide)."""
    from fractions import Fraction as F
    r = rng(4242)
    W, H = 12, 9
    for _ in range(60):
        a = r.integers(8, 8 * 11, 2)
        b = a + r.integers(-24, 25, 2)
        b = np.clip(b, 0, 8 * 11)
        # with extents (0, W, 0, H): px = x and py = H - y, both exact here
        xs = np.array([a[0] / 8, b[0] / 8])
        ys = np.array([H - min(a[1], 8 * H - 1) / 8, H - min(b[1], 8 * H - 1) / 8])
        got = o.raster(ys, (0, W, 0, H), W, H, x=xs)
        ax, bx = F(xs[0]), F(xs[1])
        ay, by = F(H) - F(ys[0]), F(H) - F(ys[1])
        for rr in range(H):
            for cc in range(W):
                for bit, sx, sy in _sample_points(cc, rr):
                    d2 = _exact_inked(sx, sy, ax, ay, bx, by)
                    if abs(d2 - 1) < F(1, 10**6):
                        continue
                    want = d2 <= 1
                    have = bool(int(got[rr, cc]) >> bit & 1)
                    assert want == have, (xs, ys, rr, cc, bit, float(d2))


def check_raster_degenerate(o):
    """No segment for fewer than two points; zero extents map to the canvas middle; a
    repeated point inks the disc of radius 1 around it (the exact test)."""
    W, H = 6, 5
    y = np.array([1.0, 2.0, 3.0])
    assert not o.raster(y, (0, 2, 0, 4), W, H, idx=np.array([1])).any()
    assert not o.raster(y[:1], (0, 2, 0, 4), W, H).any()
    # zero y extent: the line runs through the middle row (py = H/2 = 2.5)
    img = o.intensity(o.raster(np.array([7.0, 7.0]), (0, W, 7, 7), W, H, x=np.array([0.0, float(W)])))
    assert np.array_equal(img[2], np.full(W, 255, np.uint8)) and np.array_equal(img[1], np.full(W, 128, np.uint8))
    # a NaN point breaks the line: the canvas equals the two parts drawn apart
    yv = np.array([0.5, 3.0, np.nan, 1.0, 4.5])
    xv = np.array([0.0, 1.5, 3.0, 4.5, 6.0])
    both = o.raster(yv[:2], (0, W, 0, H), W, H, x=xv[:2])
    o.raster(yv[3:], (0, W, 0, H), W, H, x=xv[3:], mask=both)
    assert np.array_equal(o.raster(yv, (0, W, 0, H), W, H, x=xv), both)
    # far-away points leave the canvas untouched where the line does not pass
    far = o.raster(np.array([1e300, -1e300]), (0, W, 0, H), W, H, x=np.array([-1e300, -1e300]))
    assert not far.any()
    from fractions import Fraction as F
    got = o.raster(np.array([2.5, 2.5]), (0, W, 0, H), W, H, x=np.array([2.5, 2.5]))
    for rr in range(H):
        for cc in range(W):
            for bit, sx, sy in _sample_points(cc, rr):
                want = (sx - F(5, 2)) ** 2 + (sy - F(5, 2)) ** 2 <= 1
                assert want == bool(int(got[rr, cc]) >> bit & 1)


def check_visual_counts(o):
    """PEM/MSE counts on hand-made images: identical images differ nowhere; a 3 x 3
    blob of 255 against a blank image differs in 9 pixels by 255 and its conv-mask is
    the 5 x 5 square around it; differences of exactly the margin do not count."""
    W, H = 9, 8
    ref = np.zeros((H, W), np.uint8)
    ref[2:5, 3:6] = 255
    assert o.visual_counts(ref, ref) == (0, 0, 25)
    assert o.visual_counts(ref, np.zeros_like(ref)) == (9, 9 * 255 * 255, 25)
    img = ref.copy()
    img[3, 4] = 255 - 20
    img[2, 3] = 255 - 21
    assert o.visual_counts(ref, img) == (1, 20 * 20 + 21 * 21, 25)
    # a blob at the corner: the mask is clipped to the canvas
    ref2 = np.zeros((H, W), np.uint8)
    ref2[0, 0] = 1
    assert o.visual_counts(ref2, ref2) == (0, 0, 4)
    assert o.visual_counts(np.zeros_like(ref), ref) == (9, 9 * 255 * 255, 0)


ALL_CHECKS = [
    check_worked_examples,
    check_minmax_index_bins,
    check_minmax_xwidth_bins,
    check_preselect,
    check_lttb_exact,
    check_lttb_general,
    check_invariants,
    check_symmetries,
    check_constant_series,
    check_m4,
    check_minmax_xwidth_f64,
    check_nan_aware,
    check_raster_closed_forms,
    check_raster_brute_force,
    check_raster_degenerate,
    check_visual_counts,
]
