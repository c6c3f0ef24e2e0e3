"""The three launch paths of a single-series call (split kernels, fused persistent
tail, fully fused persistent kernel) return the oracle's result, index for index, on the same
inputs: both bin modes, float32/float64 y, implicit / int64 / float64 x, preselection,
M4, MinMaxLTTB and plain LTTB with small buckets, empty and degenerate sizes, bins
spanning several cluster CTAs and tiles, and the path the automatic choice takes."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

PATHS = ["split", "fused_tail", "fused"]


@pytest.fixture
def path(mm, request):
    yield request.param
    mm.set_single_path(mm.PATH_AUTO)


def use(mm, name):
    mm.set_single_path({"split": mm.PATH_SPLIT, "fused_tail": mm.PATH_FUSED_TAIL,
                        "fused": mm.PATH_FUSED}[name])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def walk(n, dtype, seed):
    r = np.random.default_rng(seed + 1000 * n)
    return np.cumsum(r.standard_normal(n)).astype(dtype)


def xs(n, seed, kind):
    r = np.random.default_rng(seed + 31)
    g = r.integers(0, 9, n)
    g[0] = 0
    if n > 10:
        g[r.integers(1, n, 3)] += 5000
    x = np.cumsum(g) + 123
    return x.astype(np.int64) if kind == "i64" else x.astype(np.float64) * 0.37


def eq(got, exp, what):
    got = got.cpu().numpy()
    assert np.array_equal(got, exp), f"{what}: got {got[:12]} ... expected {exp[:12]} ..."


SIZES = [0, 1, 2, 3, 5, 17, 100, 1000, 4099, 65_537, 300_007]


@pytest.mark.parametrize("path", PATHS, indirect=True)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_minmaxlttb_index_bins(mm, ref, path, n, dtype):
    use(mm, path)
    y = walk(n, dtype, 1)
    yd = dev(y)
    for n_out, r_ps in ((3, 2), (10, 4), (100, 4), (1000, 4), (4000, 2), (777, 8)):
        if n_out < n:
            eq(mm.minmaxlttb(yd, n_out, r_ps), ref.minmaxlttb(y, n_out, r_ps),
               f"{path} n={n} n_out={n_out} r_ps={r_ps}")


@pytest.mark.parametrize("path", PATHS, indirect=True)
@pytest.mark.parametrize("n", [3, 50, 1000, 65_537, 300_007])
@pytest.mark.parametrize("xkind", ["i64", "f64"])
def test_minmaxlttb_xwidth_bins(mm, ref, path, n, xkind):
    use(mm, path)
    y = walk(n, np.float64, 2)
    x = xs(n, 2, xkind)
    yd, xd = dev(y), dev(x)
    for n_out, r_ps in ((3, 4), (50, 4), (1000, 4), (3000, 2)):
        if n_out < n:
            eq(mm.minmaxlttb(yd, n_out, r_ps, x=xd, binmode=mm.BINS_XWIDTH),
               ref.minmaxlttb(y, n_out, r_ps, x=x, binmode="xwidth"),
               f"{path} xwidth {xkind} n={n} n_out={n_out}")


@pytest.mark.parametrize("path", PATHS, indirect=True)
@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 65_537])
def test_preselect_and_m4(mm, ref, path, n):
    use(mm, path)
    y = walk(n, np.float32, 3)
    yd = dev(y)
    for n_out, r_ps in ((1, 2), (5, 4), (64, 4), (2000, 4), (7, 1)):
        eq(mm.minmax_preselect(yd, n_out, r_ps), ref.minmax_preselect(y, n_out, r_ps),
           f"{path} preselect n={n} n_out={n_out} r_ps={r_ps}")
    for n_out in (4, 9, 400, 4000):
        eq(mm.m4(yd, n_out), ref.m4(y, n_out), f"{path} m4 n={n} n_out={n_out}")
    if n > 2:
        x = xs(n, 3, "i64")
        xd = dev(x)
        eq(mm.m4(yd, 40, x=xd, binmode=mm.BINS_XWIDTH), ref.m4(y, 40, x=x, binmode="xwidth"),
           f"{path} m4 xwidth n={n}")
        yn = y.copy()
        yn[::97] = np.nan
        eq(mm.minmax_preselect(dev(yn), 50, 4, nan_aware=True),
           ref.minmax_preselect(yn, 50, 4, nan_aware=True), f"{path} nan-aware n={n}")


@pytest.mark.parametrize("path", PATHS, indirect=True)
@pytest.mark.parametrize("n,n_out", [(10, 3), (1000, 400), (1000, 999), (100_000, 20_000)])
def test_plain_lttb_small_buckets(mm, ref, path, n, n_out):
    use(mm, path)
    y = walk(n, np.float64, 4)
    eq(mm.lttb(dev(y), n_out), ref.lttb(y, n_out), f"{path} lttb n={n} n_out={n_out}")


@pytest.mark.parametrize("path", PATHS, indirect=True)
def test_many_bins_across_tiles(mm, ref, path):
    """120000 bins: every CTA of the fused kernel owns more than one 512-bin tile;
    ties make argmin == argmax bins and repeated x make empty bins and ragged
    counts; 240000 table positions exceed the shared-memory staging of the chain."""
    use(mm, path)
    n = 400_003
    r = np.random.default_rng(5)
    y = r.integers(-2, 3, n).astype(np.float32)
    yd = dev(y)
    eq(mm.minmax_preselect(yd, 60000, 4), ref.minmax_preselect(y, 60000, 4), f"{path} ties")
    x = np.cumsum(r.integers(0, 3, n) * (r.random(n) < 0.3)).astype(np.int64)
    y2 = walk(n, np.float64, 6)
    eq(mm.minmaxlttb(dev(y2), 40000, 6, x=dev(x), binmode=mm.BINS_XWIDTH),
       ref.minmaxlttb(y2, 40000, 6, x=x, binmode="xwidth"), f"{path} sparse x")
    y3 = walk(n, np.float32, 8)
    eq(mm.minmaxlttb(dev(y3), 60000, 4), ref.minmaxlttb(y3, 60000, 4), f"{path} 240k positions")


def test_auto_path_choice(mm):
    sp = mm.single_path
    assert sp(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, 1_000_000, 1000) == mm.PATH_FUSED
    assert sp(mm.OP_MINMAXLTTB, mm.F64, mm.X_I64, 10**9, 4000, 4, mm.BINS_XWIDTH) == mm.PATH_FUSED_TAIL
    assert sp(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, 10**8, 200_000, 4) == mm.PATH_SPLIT  # 4e5 bins
    assert sp(mm.OP_LTTB, mm.F32, mm.X_IMPLICIT, 10**6, 1000) == mm.PATH_SPLIT  # buckets of 1000
    assert sp(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, 10, 20) == mm.PATH_SPLIT  # every index


def test_fused_is_one_launch_and_clears_status(mm, ref):
    n = 1_000_000
    y = walk(n, np.float32, 7)
    yd = dev(y)
    ws = torch.full((mm.workspace_bytes(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, n, 1000, 4),),
                    0xFF, dtype=torch.uint8, device="cuda")  # stale status bits
    before = mm.launch_count()
    got = mm.minmaxlttb(yd, 1000, 4, workspace=ws)
    assert mm.launch_count() - before == 1
    eq(got, ref.minmaxlttb(y, 1000, 4), "fused 1e6")
    assert mm.workspace_status(ws) == 0


def test_paths_agree_on_a_large_series(mm, ref):
    """2e7 float64 points, x-width bins on int64 x: the three paths give the same
    indices, and the oracle agrees."""
    n = 20_000_000
    x = synth.exp_gaps_x(n, seed=11)
    y = synth.random_walk(n, seed=11, dtype=np.float64)
    yd, xd = dev(y), dev(x)
    exp = ref.minmaxlttb(y, 4000, 4, x=x, binmode="xwidth")
    try:
        for p in PATHS:
            use(mm, p)
            eq(mm.minmaxlttb(yd, 4000, 4, x=xd, binmode=mm.BINS_XWIDTH), exp, p)
    finally:
        mm.set_single_path(mm.PATH_AUTO)
