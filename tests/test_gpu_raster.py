"""Line-chart rasterisation and the visual metrics on the GPU (mmlttb_raster,
mmlttb_raster_intensity, mmlttb_visual_counts) against the oracle, bit for bit:
sample masks of every pixel, intensities, and the integer counts behind PEM_20 and
MSE.  Cases: float32/float64 y; implicit, int64 and float64 x; all points and
selected indices; ragged canvases (one pixel, one row, one column, sides that are
not multiples of anything); zero, reversed and tight extents; long segments that
cross the whole canvas; NaN points; overlays into a non-empty canvas; a dense
1e6-point reference chart with the downsampled charts compared against it."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_mask(t):
    return t.cpu().numpy().view(np.uint32)


def extents(y, x=None):
    xs = np.arange(len(y), dtype=np.float64) if x is None else x.astype(np.float64)
    fin = y[np.isfinite(y)]
    return (float(xs[0]), float(xs[-1]), float(fin.min()), float(fin.max()))


def check(mm, ref, y, ext, w, h, x=None, idx=None, what=""):
    got = mm.raster(dev(y), ext, w, h, x=None if x is None else dev(x), idx=None if idx is None else dev(idx))
    exp = ref.raster(y, ext, w, h, x=x, idx=idx)
    g = host_mask(got)
    if not np.array_equal(g, exp):
        bad = np.argwhere(g != exp)
        r, c = bad[0]
        pytest.fail(f"{what}: {len(bad)} pixels differ, first ({r},{c}) got {g[r, c]:#06x} "
                    f"expected {exp[r, c]:#06x}")
    gi = mm.intensity(got).cpu().numpy()
    assert np.array_equal(gi, ref.intensity(exp)), f"{what}: intensity"
    return got, exp


@pytest.mark.parametrize("n", [2, 3, 17, 1000, 100_003])
@pytest.mark.parametrize("wh", [(1, 1), (1, 40), (40, 1), (37, 23), (800, 250), (257, 600)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_all_points(mm, ref, n, wh, dtype):
    y = synth.random_walk(n, seed=n, dtype=dtype)
    w, h = wh
    check(mm, ref, y, extents(y), w, h, what=f"n={n} {w}x{h} {dtype.__name__}")


@pytest.mark.parametrize("xkind", ["i64", "f64"])
def test_explicit_x(mm, ref, xkind):
    n = 20_011
    y = synth.random_walk(n, seed=3, dtype=np.float64)
    x = synth.exp_gaps_x(n, seed=3, mean_gap=50.0, big_gaps=3, big_gap=100_000)
    if xkind == "f64":
        x = x.astype(np.float64) * 0.731
    check(mm, ref, y, extents(y, x), 640, 200, x=x, what=f"x {xkind}")


@pytest.mark.parametrize("n_out", [100, 1000, 4000])
def test_selected_indices(mm, ref, n_out):
    """Charts of MinMaxLTTB, LTTB and M4 selections (the indices come from the GPU
    downsamplers; the canvas only depends on which points they name)."""
    n = 200_003
    y = synth.walk_sines_spikes(n, seed=9)
    yd = dev(y)
    ext = extents(y)
    for name, sel in (("minmaxlttb", mm.minmaxlttb(yd, n_out, 4)), ("lttb", mm.lttb(yd, n_out)),
                      ("m4", mm.m4(yd, n_out))):
        check(mm, ref, y, ext, 800, 250, idx=sel.cpu().numpy(), what=f"{name} n_out={n_out}")


def test_extents_and_degenerate_lines(mm, ref):
    y = synth.random_walk(5000, seed=4, dtype=np.float32)
    lo, hi = float(y.min()), float(y.max())
    for ext in ((0, 4999, lo, hi), (4999, 0, lo, hi), (0, 4999, hi, lo), (-1000, 6000, lo - 50, hi + 50),
                (1000, 2000, lo / 2, hi / 2), (0, 0, lo, hi), (0, 4999, 3.0, 3.0)):
        check(mm, ref, y, ext, 333, 111, what=f"extents {ext}")
    const = np.full(300, 2.5, np.float64)
    check(mm, ref, const, (0, 299, 2.5, 2.5), 120, 31, what="constant series")
    check(mm, ref, np.array([0.0, 1.0]), (0, 1, 0, 1), 1000, 700, what="one diagonal across the canvas")
    check(mm, ref, np.array([0.0, 1.0, 0.0, 1.0]), (0, 3, 0, 1), 999, 65, what="steep zigzag")
    check(mm, ref, np.array([0.0, 1.0]), (0, 1, 0, 1), 3, 40000, what="a box of 40000 rows")
    check(mm, ref, np.array([1.0, 1.0]), (0, 1, 0, 2), 50, 50, x=np.array([7, 7], np.int64),
          what="repeated point (a dot)")


def test_nan_points_and_overlay(mm, ref):
    y = synth.random_walk(3000, seed=5, dtype=np.float64)
    y[[0, 17, 18, 1500, 2999]] = np.nan
    ext = extents(y)
    check(mm, ref, y, ext, 300, 100, what="NaN points")
    # two polylines into one canvas
    y2 = synth.random_walk(3000, seed=6, dtype=np.float64)
    m = mm.raster(dev(y2), ext, 300, 100)
    mm.raster(dev(y), ext, 300, 100, mask=m)
    exp = ref.raster(y2, ext, 300, 100)
    ref.raster(y, ext, 300, 100, mask=exp)
    assert np.array_equal(host_mask(m), exp)


def test_one_launch_per_chart(mm):
    y = dev(synth.random_walk(10_000, seed=7))
    before = mm.launch_count()
    m = mm.raster(y, (0, 9999, -200, 200), 400, 100)
    assert mm.launch_count() - before == 1
    mm.intensity(m)
    assert mm.launch_count() - before == 2
    before = mm.launch_count()
    mm.raster(y[:1], (0, 1, 0, 1), 10, 10)
    assert mm.launch_count() == before  # fewer than two points: nothing enqueued


def test_visual_counts_match_oracle(mm, ref):
    r = np.random.default_rng(8)
    for h, w in ((1, 1), (1, 9), (7, 1), (31, 45), (250, 800)):
        a = (r.random((h, w)) < 0.2) * r.integers(0, 256, (h, w))
        b = np.clip(a.astype(np.int64) + r.integers(-40, 41, (h, w)) * (r.random((h, w)) < 0.5), 0, 255)
        a, b = a.astype(np.uint8), b.astype(np.uint8)
        for margin in (0, 20, 255):
            assert mm.visual_counts(dev(a), dev(b), margin) == ref.visual_counts(a, b, margin), (h, w, margin)


def test_dense_reference_and_downsampled_charts(mm, ref):
    """A 1e6-point reference chart at 800 x 250 and the charts of MinMaxLTTB (r_ps 2,
    4, 8), LTTB and M4 at n_out = 1000: canvases, intensities and the PEM_20 / MSE
    counts all equal the oracle's."""
    n = 1_000_000
    y = synth.walk_sines_spikes(n, seed=0)
    yd = dev(y)
    ext = extents(y)
    gref, eref = check(mm, ref, y, ext, 800, 250, what="reference 1e6")
    ri = mm.intensity(gref)
    ri_host = ref.intensity(eref)
    for name, sel in (("minmaxlttb2", mm.minmaxlttb(yd, 1000, 2)), ("minmaxlttb4", mm.minmaxlttb(yd, 1000, 4)),
                      ("minmaxlttb8", mm.minmaxlttb(yd, 1000, 8)), ("lttb", mm.lttb(yd, 1000)),
                      ("m4", mm.m4(yd, 1000))):
        g, e = check(mm, ref, y, ext, 800, 250, idx=sel.cpu().numpy(), what=name)
        gi = mm.intensity(g)
        assert mm.visual_counts(ri, gi, 20) == ref.visual_counts(ri_host, ref.intensity(e), 20), name
