"""GPU path vs the oracle, index array by index array (bit-exact), through the C ABI.

Small sweeps cover every branch (arange, plain LTTB, MinMax + LTTB, preselect only),
both LTTB engines (transition tables; the large-bucket fixpoint engine), both bin modes, float32 and
float64 y, implicit / int64 / float64 x, ties, signed zeros, constant series, empty
and degenerate sizes, and misaligned y pointers.  Full-size cases follow the
workloads the method is measured on."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(kind, n, seed=0):
    r = np.random.default_rng(seed * 7919 + n)
    if kind == "walk32":
        return np.cumsum(r.standard_normal(n)).astype(np.float32)
    if kind == "walk64":
        return np.cumsum(r.standard_normal(n))
    if kind == "ties32":
        return r.integers(-3, 4, n).astype(np.float32)
    if kind == "ties64":
        return r.integers(-2, 3, n).astype(np.float64)
    if kind == "zeros64":
        return np.array([-0.0, 0.0, -1.0, 1.0])[r.integers(0, 4, n)]
    if kind == "zeros32":
        return np.array([-0.0, 0.0], np.float32)[r.integers(0, 2, n)]
    if kind == "const32":
        return np.full(n, 1.5, np.float32)
    if kind == "spiky32":
        return synth.walk_sines_spikes(n, seed=seed, periods=(50.0, 700.0), spike_p=0.01)
    raise ValueError(kind)


def increasing_x(n, seed, repeats=False, big=True):
    r = np.random.default_rng(seed + 17)
    g = r.integers(0 if repeats else 1, 9, n)
    g[0] = 0
    if big and n > 10:
        g[r.integers(1, n, 3)] += 5000
    return (np.cumsum(g) + 123).astype(np.int64)


SIZES = [0, 1, 2, 3, 4, 5, 6, 7, 9, 16, 33, 100, 257, 1000, 4097, 20011, 100_003]
KINDS = ["walk32", "walk64", "ties32", "ties64", "zeros64", "zeros32", "const32", "spiky32"]


def valid_nouts(n, cands):
    """n_out values the method accepts: n_out >= 3, or n_out >= n (every index)."""
    return sorted(v for v in cands if v >= 3 or v >= n)


def eq(got, exp, what):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    if not np.array_equal(got, exp):
        d = np.nonzero(got[: min(len(got), len(exp))] != exp[: min(len(got), len(exp))])[0]
        raise AssertionError(f"{what}: len {len(got)} vs {len(exp)}, first diffs at {d[:5]}: "
                             f"got {got[d[:5]]} expected {exp[d[:5]]}")


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", KINDS)
def test_preselect_index_bins(mm, ref, n, kind):
    y = make(kind, n)
    yd = dev(y)
    for n_out, r_ps in ((1, 2), (3, 2), (5, 4), (10, 3), (64, 4), (7, 1), (1000, 4)):
        eq(mm.minmax_preselect(yd, n_out, r_ps), ref.minmax_preselect(y, n_out, r_ps),
           f"preselect n={n} {kind} n_out={n_out} r_ps={r_ps}")


@pytest.mark.parametrize("n", [3, 4, 9, 100, 1000, 20011, 100_003])
@pytest.mark.parametrize("kind", ["walk32", "walk64", "ties32", "zeros64"])
@pytest.mark.parametrize("repeats", [False, True])
def test_preselect_xwidth_bins(mm, ref, n, kind, repeats):
    y = make(kind, n)
    x = increasing_x(n, n, repeats=repeats)
    yd, xd = dev(y), dev(x)
    for n_out, r_ps in ((1, 2), (3, 2), (8, 4), (50, 4), (333, 2)):
        eq(mm.minmax_preselect(yd, n_out, r_ps, x=xd, binmode="xwidth"),
           ref.minmax_preselect(y, n_out, r_ps, x=x, binmode="xwidth"),
           f"xwidth preselect n={n} {kind} rep={repeats} n_out={n_out}")


@pytest.mark.parametrize("n", [3, 4, 5, 10, 33, 257, 4097, 100_003])
@pytest.mark.parametrize("kind", ["walk32", "walk64", "ties32", "zeros64", "const32"])
def test_lttb(mm, ref, n, kind):
    y = make(kind, n)
    yd = dev(y)
    for n_out in valid_nouts(n, {3, 4, 5, 10, n // 3, n // 31, n // 40, n - 1, n, n + 3}):
        eq(mm.lttb(yd, n_out), ref.lttb(y, n_out), f"lttb n={n} {kind} n_out={n_out}")


@pytest.mark.parametrize("n", [3, 7, 100, 4097, 100_003])
@pytest.mark.parametrize("kind", ["walk32", "walk64", "ties64"])
def test_lttb_explicit_x(mm, ref, n, kind):
    y = make(kind, n)
    x = increasing_x(n, 5, repeats=False)
    xf = x.astype(np.float64) * 0.25
    for n_out in sorted({3, 10, max(3, n // 5), max(3, n // 100)}):
        eq(mm.lttb(dev(y), n_out, x=dev(x)), ref.lttb(y, n_out, x=x), f"lttb i64 x n={n}")
        eq(mm.lttb(dev(y), n_out, x=dev(xf)), ref.lttb(y, n_out, x=xf), f"lttb f64 x n={n}")


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 8, 13, 100, 1000, 4097, 20011, 100_003])
@pytest.mark.parametrize("kind", KINDS)
def test_minmaxlttb_index_bins(mm, ref, n, kind):
    y = make(kind, n)
    yd = dev(y)
    for n_out in valid_nouts(n, {3, 4, 7, 25, 100, n // 9, n - 1, n + 1}):
        for r_ps in (2, 3, 4, 8, 16):
            eq(mm.minmaxlttb(yd, n_out, r_ps), ref.minmaxlttb(y, n_out, r_ps),
               f"minmaxlttb n={n} {kind} n_out={n_out} r_ps={r_ps}")


@pytest.mark.parametrize("n", [5, 64, 1000, 20011, 100_003])
@pytest.mark.parametrize("kind", ["walk32", "walk64", "ties64", "zeros32"])
@pytest.mark.parametrize("repeats", [False, True])
def test_minmaxlttb_xwidth_bins(mm, ref, n, kind, repeats):
    y = make(kind, n)
    x = increasing_x(n, 3 * n, repeats=repeats)
    yd, xd = dev(y), dev(x)
    for n_out in sorted({3, 4, 10, 100, max(3, n // 7)}):
        for r_ps in (2, 4, 6):
            eq(mm.minmaxlttb(yd, n_out, r_ps, x=xd, binmode="xwidth"),
               ref.minmaxlttb(y, n_out, r_ps, x=x, binmode="xwidth"),
               f"xwidth minmaxlttb n={n} {kind} rep={repeats} n_out={n_out} r_ps={r_ps}")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("offset", [1, 2, 3, 5])
def test_misaligned_y(mm, ref, dtype, offset):
    n = 50_000 + offset
    big = make("walk64", n + 16).astype(dtype)
    bd = dev(big)
    y = big[offset: offset + n]
    yd = bd[offset: offset + n]
    eq(mm.minmax_preselect(yd, 300, 4), ref.minmax_preselect(y, 300, 4), "misaligned preselect")
    eq(mm.minmaxlttb(yd, 500, 4), ref.minmaxlttb(y, 500, 4), "misaligned minmaxlttb")
    x = increasing_x(n, 11)
    eq(mm.minmaxlttb(yd, 400, 4, x=dev(x), binmode="xwidth"),
       ref.minmaxlttb(y, 400, 4, x=x, binmode="xwidth"), "misaligned xwidth")


def test_large_bucket_means_exact_and_fallback(mm, ref):
    """Next-bucket means of large buckets (grid engine; one CTA per series in a
    batch): integer-valued y, whose sums are exact in any order (the lanes add in
    parallel), y whose magnitudes span 2^-60..2^60 in every bucket (the sums round:
    one lane adds left to right), float32 y, and signed zeros all equal the oracle."""
    r = np.random.default_rng(12)
    n = 200_003
    yi = np.cumsum(r.integers(-3, 4, n)).astype(np.float64)
    ys = r.standard_normal(n) * 2.0 ** r.integers(-60, 61, n)
    yz = np.where(r.random(n) < 0.5, -0.0, 0.0)
    yz[::1001] = 1.0
    series = [("int", yi), ("span", ys), ("span32", ys.astype(np.float32)), ("zeros", yz)]
    for name, y in series:
        for n_out in (40, 300):
            eq(mm.lttb(dev(y), n_out), ref.lttb(y, n_out), f"grid lttb {name} n_out={n_out}")
    b = mm.Batch([{"y": dev(y), "n_out": 40, "op": "lttb"} for _, y in series])
    b.run()
    for (name, y), got in zip(series, b.results()):
        eq(got, ref.lttb(y, 40), f"block lttb {name}")


def test_table_engine_threshold(mm, ref):
    """Bucket sizes around the transition-table limit (32 points)."""
    y = make("walk64", 10_000, seed=5)
    for n_out in (2 + (10_000 - 2) // 32, 2 + (10_000 - 2) // 33, 2 + (10_000 - 2) // 31, 300, 301):
        eq(mm.lttb(dev(y), n_out), ref.lttb(y, n_out), f"lttb threshold n_out={n_out}")


def test_grid_engine_large_buckets(mm, ref):
    """Plain LTTB with buckets of ~1e4..5e5 points (the large-bucket fixpoint engine)."""
    y = synth.random_walk(1_000_003, seed=9, dtype=np.float32)
    yd = dev(y)
    for n_out in (3, 4, 100, 1000):
        eq(mm.lttb(yd, n_out), ref.lttb(y, n_out), f"grid lttb n_out={n_out}")
    y64 = synth.random_walk(300_001, seed=10, dtype=np.float64)
    x = increasing_x(300_001, 2)
    eq(mm.lttb(dev(y64), 50, x=dev(x)), ref.lttb(y64, 50, x=x), "grid lttb f64 x")
    # MinMaxLTTB whose preselected buckets exceed the table limit (r_ps = 80)
    eq(mm.minmaxlttb(yd, 50, 80), ref.minmaxlttb(y, 50, 80), "grid minmaxlttb r_ps=80")


def test_workspace_status_and_reuse(mm, ref):
    y = make("walk32", 200_000)
    yd = dev(y)
    ws = torch.empty(mm.workspace_bytes(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, 200_000, 2000, 4),
                     dtype=torch.uint8, device="cuda")
    for n_out in (2000, 100, 1500):
        eq(mm.minmaxlttb(yd, n_out, 4, workspace=ws), ref.minmaxlttb(y, n_out, 4), "reuse")
    assert mm.workspace_status(ws) == 0
    wsl = torch.empty(mm.workspace_bytes(mm.OP_LTTB, mm.F32, mm.X_IMPLICIT, 200_000, 10),
                      dtype=torch.uint8, device="cuda")
    eq(mm.lttb(yd, 10, workspace=wsl), ref.lttb(y, 10), "grid lttb")
    assert mm.workspace_status(wsl) == 0


def test_workspace_too_small_and_bad_args(mm):
    y = dev(make("walk32", 1000))
    with pytest.raises(mm.MMLTTBError) as e:
        mm.minmaxlttb(y, 100, 4, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert e.value.code == mm.ENOSPC
    with pytest.raises(mm.MMLTTBError) as e:
        mm.minmaxlttb(y, 2, 4)
    assert e.value.code == mm.EINVAL


def test_side_stream(mm, ref):
    y = make("walk64", 300_000, seed=4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        yd = dev(y)
        got = mm.minmaxlttb(yd, 1234, 4)
    s.synchronize()
    eq(got, ref.minmaxlttb(y, 1234, 4), "side stream")


# ---------------------------------------------------------------- full-size workloads
def test_single_series_1e6(mm, ref):
    """n_in = 1e6 float32 Gaussian random walk (seed 0), n_out = 1000, r_ps = 4."""
    y = synth.random_walk(1_000_000, seed=0, dtype=np.float32)
    got = mm.minmaxlttb(dev(y), 1000, 4)
    eq(got, ref.minmaxlttb(y, 1000, 4), "1e6 minmaxlttb")
    assert len(got) == 1000


@pytest.mark.slow
def test_single_series_1e8_vs_plain_lttb(mm, ref):
    """n_in = 1e8 float32 walk + sines + spikes, n_out = 2000, r_ps in {2,4,8,16}, and
    plain LTTB on all points."""
    y = synth.walk_sines_spikes(100_000_000, seed=0)
    yd = dev(y)
    for r_ps in (2, 4, 8, 16):
        eq(mm.minmaxlttb(yd, 2000, r_ps), ref.minmaxlttb(y, 2000, r_ps), f"1e8 r_ps={r_ps}")
    eq(mm.lttb(yd, 2000), ref.lttb(y, 2000), "1e8 plain lttb")


@pytest.mark.slow
def test_single_series_1e9_xwidth(mm, ref):
    """n_in = 1e9, int64 x with exponential gaps (mean 1000) and 5 gaps of 1e9,
    float64 random walk, n_out = 4000, r_ps = 4, x-width bins (16 GB input)."""
    n = 1_000_000_000
    y = synth.random_walk(n, seed=0, dtype=np.float64)
    x = synth.exp_gaps_x(n, seed=0)
    yd, xd = dev(y), dev(x)
    got = mm.minmaxlttb(yd, 4000, 4, x=xd, binmode="xwidth")
    pre = mm.minmax_preselect(yd, 4000, 4, x=xd, binmode="xwidth")
    del yd, xd
    torch.cuda.empty_cache()
    eq(pre, ref.minmax_preselect(y, 4000, 4, x=x, binmode="xwidth"), "1e9 preselect")
    eq(got, ref.minmaxlttb(y, 4000, 4, x=x, binmode="xwidth"), "1e9 minmaxlttb")


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_point(mm, ref, pinned):
    """mmlttb_minmaxlttb_host: pinned host inputs are read in place (zero-copy),
    pageable ones are staged; both equal the device entry point and the oracle."""
    n = 3_000_001
    y = synth.random_walk(n, seed=21, dtype=np.float64)
    x = synth.exp_gaps_x(n, seed=21, mean_gap=100.0, big_gaps=3, big_gap=10**8)
    yh, xh = torch.from_numpy(y), torch.from_numpy(x)
    if pinned:
        yh, xh = yh.pin_memory(), xh.pin_memory()
    for n_out, r_ps, bm, xx in ((2000, 4, "xwidth", xh), (700, 6, "index", None)):
        got = mm.minmaxlttb_host(yh, n_out, r_ps, x=xx, binmode=bm).numpy()
        exp = ref.minmaxlttb(y, n_out, r_ps, x=x if xx is not None else None, binmode=bm)
        eq(got, exp, f"host entry pinned={pinned} {bm}")
        dev_res = mm.minmaxlttb(dev(y), n_out, r_ps, x=dev(x) if xx is not None else None, binmode=bm)
        eq(dev_res, exp, "device entry")


def test_host_series_need_no_device_copy(mm, ref):
    """Pinned inputs run with the in-place device buffer, which holds no copy of the
    series (so a series may exceed device memory); pageable inputs need the staging
    size and get MMLTTB_ENOSPC (-2) with the smaller buffer."""
    n = 20_000_003
    y = synth.random_walk(n, seed=22, dtype=np.float64)
    x = synth.exp_gaps_x(n, seed=22, mean_gap=10.0, big_gaps=2, big_gap=10**7)
    yh, xh = torch.from_numpy(y).pin_memory(), torch.from_numpy(x).pin_memory()
    small = mm.host_buffer_bytes(mm.F64, mm.X_I64, n, 4000, 4, mm.BINS_XWIDTH, inplace=True)
    full = mm.host_buffer_bytes(mm.F64, mm.X_I64, n, 4000, 4, mm.BINS_XWIDTH)
    assert small < n * 8 // 4 and full >= small + 16 * n
    buf = torch.empty(small, dtype=torch.uint8, device="cuda")
    got = mm.minmaxlttb_host(yh, 4000, 4, x=xh, binmode="xwidth", device_buffer=buf).numpy()
    eq(got, ref.minmaxlttb(y, 4000, 4, x=x, binmode="xwidth"), "in place")
    with pytest.raises(mm.MMLTTBError) as e:
        mm.minmaxlttb_host(torch.from_numpy(y), 4000, 4, x=torch.from_numpy(x), binmode="xwidth",
                           device_buffer=buf)
    assert e.value.code == -2


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 100, 4097, 100_003])
@pytest.mark.parametrize("kind", ["walk32", "walk64", "ties32", "zeros64", "const32"])
def test_m4_index_bins(mm, ref, n, kind):
    y = make(kind, n)
    yd = dev(y)
    for n_out in (4, 5, 8, 100, 4 * n + 4, 1001):
        eq(mm.m4(yd, n_out), ref.m4(y, n_out), f"m4 n={n} {kind} n_out={n_out}")


@pytest.mark.parametrize("n", [2, 9, 1000, 100_003])
@pytest.mark.parametrize("repeats", [False, True])
def test_m4_xwidth_bins(mm, ref, n, repeats):
    y = make("walk64", n)
    x = increasing_x(n, 7 * n, repeats=repeats)
    for n_out in (4, 12, 400, 4000):
        eq(mm.m4(dev(y), n_out, x=dev(x), binmode="xwidth"),
           ref.m4(y, n_out, x=x, binmode="xwidth"), f"m4 xwidth n={n} n_out={n_out}")


@pytest.mark.parametrize("n", [3, 50, 20011, 100_003])
def test_xwidth_bins_float64_x(mm, ref, n):
    """Equal-width bins on float64 x (edges rounded in FP64, R17)."""
    r = np.random.default_rng(n)
    g = r.exponential(0.37, n)
    g[0] = 0.0
    g[r.integers(1, n, max(1, n // 7))] = 0.0
    if n > 10:
        g[r.integers(1, n, 2)] += 1000.0
    x = np.cumsum(g) - 11.5
    xg = np.arange(n, dtype=np.float64) * 0.5  # grid: edges land on points
    for y in (make("walk32", n), make("walk64", n), make("ties32", n)):
        for xx in (x, xg):
            for n_out, r_ps in ((3, 2), (40, 4), (1000, 4)):
                eq(mm.minmax_preselect(dev(y), n_out, r_ps, x=dev(xx), binmode="xwidth"),
                   ref.minmax_preselect(y, n_out, r_ps, x=xx, binmode="xwidth"), f"f64x preselect n={n}")
                eq(mm.minmaxlttb(dev(y), n_out, r_ps, x=dev(xx), binmode="xwidth"),
                   ref.minmaxlttb(y, n_out, r_ps, x=xx, binmode="xwidth"), f"f64x minmaxlttb n={n}")
            eq(mm.m4(dev(y), 400, x=dev(xx), binmode="xwidth"), ref.m4(y, 400, x=xx, binmode="xwidth"), "f64x m4")


@pytest.mark.parametrize("n", [3, 10, 4097, 100_003])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nan_aware_preselect_and_m4(mm, ref, n, dtype):
    """NaN-aware MinMax and M4 (R18): a bin holding NaN reports its first NaN."""
    r = np.random.default_rng(n)
    y = np.cumsum(r.standard_normal(n)).astype(dtype)
    y[r.integers(0, n, max(1, n // 50))] = np.nan
    y[r.integers(0, n, 3)] = np.inf
    x = increasing_x(n, n + 5, repeats=True)
    yd, xd = dev(y), dev(x)
    for n_out, r_ps in ((3, 2), (40, 4), (1000, 4)):
        eq(mm.minmax_preselect(yd, n_out, r_ps, nan_aware=True),
           ref.minmax_preselect(y, n_out, r_ps, nan_aware=True), f"nan preselect n={n}")
        eq(mm.minmax_preselect(yd, n_out, r_ps, x=xd, binmode="xwidth", nan_aware=True),
           ref.minmax_preselect(y, n_out, r_ps, x=x, binmode="xwidth", nan_aware=True), "nan preselect x")
    for n_out in (4, 400, 4000):
        eq(mm.m4(yd, n_out, nan_aware=True), ref.m4(y, n_out, nan_aware=True), f"nan m4 n={n}")
    with pytest.raises(mm.MMLTTBError):  # NaN-aware is for the aggregations only
        mm.minmaxlttb(yd, 100, 4, binmode=mm.BINS_INDEX | mm.NAN_AWARE)
