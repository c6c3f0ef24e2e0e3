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
