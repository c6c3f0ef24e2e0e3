"""Stream-kernel variants and the autotuner: every compiled variant gives the
oracle's indices (index and x-width bins, float32 and float64, batches), and
mmlttb_autotune selects one of them and keeps it for the process."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_every_variant_matches_oracle(mm, ref):
    variants = mm.stream_variants()
    assert len(variants) >= 2
    y32 = synth.random_walk(2_000_003, seed=31, dtype=np.float32)
    y64 = synth.random_walk(1_000_003, seed=32, dtype=np.float64)
    x64 = synth.exp_gaps_x(1_000_003, seed=32, mean_gap=30.0, big_gaps=3, big_gap=10**6)
    ties = np.random.default_rng(33).integers(-2, 3, 500_000).astype(np.float32)
    d32, d64, dx, dt = (torch.from_numpy(a).cuda() for a in (y32, y64, x64, ties))
    before = {yd: None for yd in (mm.F32, mm.F64)}
    for v in range(len(variants)):
        for yd in (mm.F32, mm.F64):
            assert mm.lib.mmlttb_set_stream_variant(yd, v) == mm.OK
        for n_out, r_ps in ((1000, 4), (3000, 8), (37, 2), (20000, 4)):
            assert np.array_equal(mm.minmaxlttb(d32, n_out, r_ps).cpu().numpy(),
                                  ref.minmaxlttb(y32, n_out, r_ps)), (v, n_out)
            assert np.array_equal(mm.minmaxlttb(dt, n_out, r_ps).cpu().numpy(),
                                  ref.minmaxlttb(ties, n_out, r_ps)), (v, n_out)
            assert np.array_equal(mm.minmaxlttb(d64, n_out, r_ps, x=dx, binmode="xwidth").cpu().numpy(),
                                  ref.minmaxlttb(y64, n_out, r_ps, x=x64, binmode="xwidth")), (v, n_out)
        assert np.array_equal(mm.m4(d64, 4000).cpu().numpy(), ref.m4(y64, 4000)), v
        b = mm.Batch([{"y": d32[: 1000 * (k + 1) ** 3], "n_out": 200 + 37 * k, "r_ps": 4} for k in range(12)])
        b.run()
        for k, r in enumerate(b.results()):
            assert np.array_equal(r.cpu().numpy(), ref.minmaxlttb(y32[: 1000 * (k + 1) ** 3], 200 + 37 * k, 4)), (v, k)
        b.close()
    for yd in (mm.F32, mm.F64):
        assert mm.lib.mmlttb_set_stream_variant(yd, 0) == mm.OK


def test_autotune_picks_a_variant(mm, tmp_path, monkeypatch):
    monkeypatch.setenv("MMLTTB_TUNE_CACHE", str(tmp_path / "tune.json"))
    y = torch.from_numpy(synth.random_walk(20_000_000, seed=34, dtype=np.float32)).cuda()
    v, ms = mm.autotune(y, n_out=4000, r_ps=4)
    assert 0 <= v < len(mm.stream_variants()) and ms > 0.0
    import ctypes
    got = ctypes.c_int(-1)
    assert mm.lib.mmlttb_get_stream_variant(mm.F32, ctypes.byref(got)) == mm.OK and got.value == v
    assert mm.load_tuning() == {"f32": v}
    assert mm.lib.mmlttb_set_stream_variant(mm.F32, 0) == mm.OK


def _mixed_tuning_batch():
    """Float32 index-bin series (the batch's key) of many sizes, plus float64 x-width
    and plain-LTTB series."""
    r = np.random.default_rng(40)
    series = []
    for i in range(24):
        n = int(10 ** r.uniform(3, 6.3))
        series.append({"y_h": synth.random_walk(n, seed=400 + i, dtype=np.float32),
                       "n_out": int(r.integers(50, 3000)), "r_ps": int(r.choice([2, 4, 8]))})
    x = synth.exp_gaps_x(300_001, seed=41, mean_gap=20.0, big_gaps=2, big_gap=10**5)
    series.append({"y_h": synth.random_walk(300_001, seed=42, dtype=np.float64), "x_h": x,
                   "n_out": 900, "r_ps": 4, "binmode": "xwidth"})
    series.append({"y_h": synth.random_walk(5000, seed=43, dtype=np.float32), "n_out": 700, "r_ps": 4,
                   "op": "lttb"})
    return series


def test_every_tuple_matches_oracle_on_a_mixed_batch(mm, ref):
    """Every tuning tuple (variant x lanes-per-bin shift x k_tables rounds) set for the
    batch's key plans the batch with that tuple and returns the oracle's indices."""
    series = _mixed_tuning_batch()
    spec, exp = [], []
    for s in series:
        d = {"y": torch.from_numpy(s["y_h"]).cuda(), "n_out": s["n_out"], "r_ps": s["r_ps"],
             "op": s.get("op", "minmaxlttb")}
        if "x_h" in s:
            d["x"] = torch.from_numpy(s["x_h"]).cuda()
            d["binmode"] = s["binmode"]
        spec.append(d)
        if d["op"] == "lttb":
            exp.append(ref.lttb(s["y_h"], s["n_out"]))
        else:
            exp.append(ref.minmaxlttb(s["y_h"], s["n_out"], s["r_ps"], x=s.get("x_h"),
                                      binmode=s.get("binmode", "index")))
    binned = sum(len(s["y_h"]) for s in series if s.get("op", "minmaxlttb") != "lttb")
    try:
        for v in range(len(mm.stream_variants())):
            for g in (-1, 0, 1):
                for rounds in (0, 1, 3, 7):
                    mm.clear_tunings()
                    mm.set_tuning(mm.F32, mm.X_IMPLICIT, mm.BINS_INDEX, binned, v, g, rounds)
                    b = mm.Batch(spec)
                    assert b.tuning() == {"variant": v, "group_shift": g, "tab_rounds": rounds}
                    b.run(graph=(rounds == 3))
                    for i, r in enumerate(b.results()):
                        assert np.array_equal(r.cpu().numpy(), exp[i]), (v, g, rounds, i)
                    b.close()
    finally:
        mm.clear_tunings()


def test_autotune_tuple_keys_and_cache(mm, ref, tmp_path, monkeypatch):
    monkeypatch.setenv("MMLTTB_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = 20_000_003
    y_h = synth.random_walk(n, seed=44, dtype=np.float32)
    y = torch.from_numpy(y_h).cuda()
    try:
        t, ms = mm.autotune_tuple(y, n_out=4000, r_ps=4)
        assert 0 <= t["variant"] < len(mm.stream_variants()) and t["group_shift"] in (-1, 0, 1)
        assert t["tab_rounds"] in (0, 2, 4, 7) and ms > 0.0
        assert mm.get_tuning(mm.F32, mm.X_IMPLICIT, mm.BINS_INDEX, n) == t
        # another size class or key keeps the default
        assert mm.get_tuning(mm.F32, mm.X_IMPLICIT, mm.BINS_INDEX, n // 100)["group_shift"] == 0
        assert np.array_equal(mm.minmaxlttb(y, 4000, 4).cpu().numpy(), ref.minmaxlttb(y_h, 4000, 4))
        mm.clear_tunings()
        applied = mm.load_tuning()
        assert t in applied.values()
        assert mm.get_tuning(mm.F32, mm.X_IMPLICIT, mm.BINS_INDEX, n) == t
    finally:
        mm.clear_tunings()


def test_autotune_batch_keeps_the_fastest_tuple(mm, ref):
    series = _mixed_tuning_batch()[:12]
    spec = [{"y": torch.from_numpy(s["y_h"]).cuda(), "n_out": s["n_out"], "r_ps": s["r_ps"]} for s in series]
    try:
        best, ms, timings = mm.autotune_batch(spec, steps=3, warmup=1, shifts=(0, 1), rounds=(0, 4))
        assert len(timings) == len(mm.stream_variants()) * 4 and ms == min(timings.values())
        b = mm.Batch(spec)
        assert b.tuning() == best
        b.run(graph=True)
        for i, r in enumerate(b.results()):
            assert np.array_equal(r.cpu().numpy(), ref.minmaxlttb(series[i]["y_h"], series[i]["n_out"],
                                                                   series[i]["r_ps"])), i
        b.close()
    finally:
        mm.clear_tunings()
