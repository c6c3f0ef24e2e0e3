"""The staged MinMax stream (tiles of whole bins of float32 y copied into shared
memory by cp.async.bulk) against the oracle, element by element, and against the
register stream: index bins from 1 to 128 points (float64 y, which takes the register
stream, alongside), ties, a y pointer off a 16-byte boundary, NaN-aware
bins, M4, empty bins, full MinMaxLTTB, and batches that mix staged, register-streamed
and x-width series."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

# launches of at least 64 MiB of y take the staged stream for small index bins
N32 = 17_000_003
N64 = 8_500_003


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def walk(n, seed, dt):
    return synth.random_walk(n, seed=seed, dtype=dt)


def n_out_for(n, S, r_ps=2):
    """n_out giving bins of about S points (B = n_out * r_ps / 2 bins)."""
    B = max(1, int((n - 2) / S))
    return max(3, (2 * B) // r_ps)


def staged(mm, op, y, n_out, r_ps, binmode=0):
    yd = mm.F32 if y.dtype == np.float32 else mm.F64
    return mm.stream_tiles(op, yd, mm.X_IMPLICIT, len(y), n_out, r_ps, binmode)


@pytest.fixture(autouse=True)
def staging_on(mm):
    """The staged stream is opt-in: on for every test here, off again afterwards."""
    mm.set_stream_staging(True)
    yield
    mm.set_stream_staging(False)


@pytest.fixture
def register_stream(mm):
    """Run a block with the staged stream off; on again afterwards."""
    class Ctx:
        def __enter__(self):
            mm.set_stream_staging(False)

        def __exit__(self, *a):
            mm.set_stream_staging(True)
    return Ctx()


@pytest.mark.parametrize("dt,S", [(np.float32, 1.3), (np.float32, 3), (np.float32, 16), (np.float32, 16.5),
                                  (np.float32, 64), (np.float32, 100), (np.float32, 127),
                                  (np.float64, 1.5), (np.float64, 17), (np.float64, 60)])
def test_staged_preselect_matches_oracle(mm, ref, register_stream, dt, S):
    n = N32 if dt == np.float32 else N64
    y_h = walk(n, 11, dt)
    n_out = n_out_for(n, S)
    # float64 y takes the register stream
    assert (staged(mm, mm.OP_PRESELECT, y_h, n_out, 2) > 0) == (dt == np.float32)
    y = dev(y_h)
    got = mm.minmax_preselect(y, n_out, 2).cpu().numpy()
    assert np.array_equal(got, ref.minmax_preselect(y_h, n_out, 2)), (dt, S)
    with register_stream:
        assert staged(mm, mm.OP_PRESELECT, y_h, n_out, 2) == 0
        reg = mm.minmax_preselect(y, n_out, 2).cpu().numpy()
    assert np.array_equal(got, reg)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_staged_ties_first_occurrence(mm, ref, dt):
    """Integer-valued y in [-2, 2]: every bin has many tied extremes."""
    n = N32 if dt == np.float32 else N64
    y_h = np.random.default_rng(5).integers(-2, 3, n).astype(dt)
    for S in (7, 64, 120):
        n_out = n_out_for(n, S)
        assert (staged(mm, mm.OP_PRESELECT, y_h, n_out, 2) > 0) == (dt == np.float32)
        got = mm.minmax_preselect(dev(y_h), n_out, 2).cpu().numpy()
        assert np.array_equal(got, ref.minmax_preselect(y_h, n_out, 2)), (dt, S)


@pytest.mark.parametrize("dt,off", [(np.float32, 1), (np.float32, 2), (np.float32, 3), (np.float64, 1)])
def test_staged_unaligned_pointer(mm, ref, dt, off):
    """y starting 4, 8 or 12 bytes past a 16-byte boundary (a view into a larger
    tensor): the first and last tiles' copies start and end on the boundaries around
    the series, inside the allocation."""
    n = (N32 if dt == np.float32 else N64) - 7
    base_h = walk(n + off + 5, 12, dt)
    base = dev(base_h)
    y = base[off:off + n]
    assert y.data_ptr() % 16 != 0
    y_h = base_h[off:off + n]
    for S in (5, 100):
        n_out = n_out_for(n, S)
        assert (staged(mm, mm.OP_PRESELECT, y_h, n_out, 2) > 0) == (dt == np.float32)
        got = mm.minmax_preselect(y, n_out, 2).cpu().numpy()
        assert np.array_equal(got, ref.minmax_preselect(y_h, n_out, 2)), (dt, off, S)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_staged_nan_aware(mm, ref, dt):
    n = N32 if dt == np.float32 else N64
    y_h = walk(n, 13, dt)
    r = np.random.default_rng(14)
    y_h[r.integers(0, n, 2000)] = np.nan
    y_h[1:40] = np.nan  # the whole first bins
    for S in (9, 120):
        n_out = n_out_for(n, S)
        assert (staged(mm, mm.OP_PRESELECT, y_h, n_out, 2) > 0) == (dt == np.float32)
        got = mm.minmax_preselect(dev(y_h), n_out, 2, nan_aware=True).cpu().numpy()
        assert np.array_equal(got, ref.minmax_preselect(y_h, n_out, 2, nan_aware=True)), (dt, S)


def test_staged_m4(mm, ref):
    y_h = walk(N32, 15, np.float32)
    for S in (6, 120):
        n_out = 4 * max(1, int(N32 / S))
        assert staged(mm, mm.OP_M4, y_h, n_out, 4) > 0
        got = mm.m4(dev(y_h), n_out).cpu().numpy()
        assert np.array_equal(got, ref.m4(y_h, n_out)), S


@pytest.mark.parametrize("r_ps", [2, 4, 8])
def test_staged_minmaxlttb(mm, ref, r_ps):
    y_h = walk(N32, 16, np.float32)
    n_out = 150_000
    assert staged(mm, mm.OP_MINMAXLTTB, y_h, n_out, r_ps) > 0
    got = mm.minmaxlttb(dev(y_h), n_out, r_ps).cpu().numpy()
    assert np.array_equal(got, ref.minmaxlttb(y_h, n_out, r_ps)), r_ps


def test_staged_mixed_batch(mm, ref, register_stream):
    """One batch over 64 MiB: staged float32 series (small bins), register-streamed ones
    (float64 y, bins over 512 bytes), x-width bins, series with more bins than
    points (empty bins), M4 and tiny series; the same batch with the staged stream
    off gives the same indices."""
    r = np.random.default_rng(17)
    series = [
        {"y_h": walk(9_000_001, 20, np.float32), "n_out": 600_000, "r_ps": 2, "op": "preselect"},
        {"y_h": walk(3_000_017, 21, np.float64), "n_out": 40_000, "r_ps": 4, "op": "minmaxlttb"},
        {"y_h": walk(4_000_003, 22, np.float32), "n_out": 300, "r_ps": 2, "op": "preselect"},
        {"y_h": walk(2_000_000, 23, np.float32), "n_out": 20_000, "r_ps": 4, "op": "minmaxlttb"},
        {"y_h": walk(1000, 24, np.float32), "n_out": 700, "r_ps": 4, "op": "preselect"},
        {"y_h": walk(5, 25, np.float64), "n_out": 4, "r_ps": 2, "op": "preselect"},
        {"y_h": walk(1_000_000, 26, np.float32), "n_out": 40_000, "r_ps": 4, "op": "m4"},
    ]
    g = r.integers(1, 4, 600_000)
    g[0] = 0
    series.append({"y_h": walk(600_000, 27, np.float32), "x_h": np.cumsum(g).astype(np.int64),
                   "n_out": 1000, "r_ps": 4, "op": "minmaxlttb", "binmode": "xwidth"})
    spec = []
    for s in series:
        d = {"y": dev(s["y_h"]), "n_out": s["n_out"], "r_ps": s["r_ps"], "op": s["op"]}
        if "x_h" in s:
            d["x"] = dev(s["x_h"])
            d["binmode"] = s["binmode"]
        spec.append(d)

    def expect(s):
        x, bm = s.get("x_h"), s.get("binmode", "index")
        if s["op"] == "preselect":
            return ref.minmax_preselect(s["y_h"], s["n_out"], s["r_ps"], x=x, binmode=bm)
        if s["op"] == "m4":
            return ref.m4(s["y_h"], s["n_out"], x=x, binmode=bm)
        return ref.minmaxlttb(s["y_h"], s["n_out"], s["r_ps"], x=x, binmode=bm)

    exp = [expect(s) for s in series]
    b = mm.Batch(spec)
    for graph in (False, True):
        b.run(graph=graph)
        res = b.results()
        for i in range(len(series)):
            assert np.array_equal(res[i].cpu().numpy(), exp[i]), (i, graph)
    b.close()
    with register_stream:
        b = mm.Batch(spec)
        b.run(graph=False)
        res = b.results()
        for i in range(len(series)):
            assert np.array_equal(res[i].cpu().numpy(), exp[i]), ("register", i)
        b.close()


def test_staging_toggle(mm):
    assert mm.stream_staging()  # on (fixture); off is the library's default
    y = np.zeros(N32, np.float32)
    assert staged(mm, mm.OP_PRESELECT, y, n_out_for(N32, 100), 2) > 0
    # below 64 MiB, and bins over 512 bytes, take the register stream
    assert staged(mm, mm.OP_PRESELECT, y[: N32 // 4], n_out_for(N32 // 4, 100), 2) == 0
    assert staged(mm, mm.OP_PRESELECT, y, n_out_for(N32, 5000), 2) == 0
    mm.set_stream_staging(False)
    try:
        assert not mm.stream_staging()
        assert staged(mm, mm.OP_PRESELECT, y, n_out_for(N32, 100), 2) == 0
    finally:
        mm.set_stream_staging(True)
