"""Batched path vs the oracle: every series of a mixed batch (lengths, dtypes, x
kinds, bin modes, ops, n_out, r_ps) equals the oracle's result, with and without a
CUDA graph, and a graph replay picks up new data in the same buffers."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_result(ref, s):
    y = s["y_h"]
    x = s.get("x_h")
    op = s.get("op", "minmaxlttb")
    if op == "lttb":
        return ref.lttb(y, s["n_out"], x=x)
    if op == "m4":
        return ref.m4(y, s["n_out"], x=x, binmode=s.get("binmode", "index"))
    if op == "preselect":
        return ref.minmax_preselect(y, s["n_out"], s.get("r_ps", 4), x=x, binmode=s.get("binmode", "index"))
    return ref.minmaxlttb(y, s["n_out"], s.get("r_ps", 4), x=x, binmode=s.get("binmode", "index"))


def mixed_series(seed, count):
    r = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(r.choice([0, 1, 2, 3, 5, 17, 100, 1000, 5000, 30_000, 120_000, 400_000]))
        dt = np.float32 if r.random() < 0.6 else np.float64
        y = np.cumsum(r.standard_normal(n)).astype(dt) if r.random() < 0.8 else \
            r.integers(-3, 4, n).astype(dt)
        s = {"y_h": y, "n_out": int(r.choice([3, 4, 10, 57, 200, 1000, 4000])),
             "r_ps": int(r.choice([2, 3, 4, 8])),
             "op": str(r.choice(["minmaxlttb", "minmaxlttb", "lttb", "preselect", "m4"]))}
        if s["op"] == "m4":
            s["n_out"] = max(4, s["n_out"])  # M4 takes n_out >= 4
        if s["op"] == "lttb" and n > s["n_out"] and (n - 2) // max(1, s["n_out"] - 2) > 2000:
            s["n_out"] = max(3, n // 1000)  # keep plain-LTTB buckets modest in a batch
        if n >= 3 and r.random() < 0.4:
            g = r.integers(1, 5, n)
            g[0] = 0
            if n > 10:
                g[r.integers(1, n)] += 10_000
            s["x_h"] = np.cumsum(g).astype(np.int64)
            if s["op"] != "lttb" and r.random() < 0.7:
                s["binmode"] = "xwidth"
        out.append(s)
    return out


def to_batch(mm, series):
    spec = []
    for s in series:
        d = {"y": dev(s["y_h"]), "n_out": s["n_out"], "r_ps": s["r_ps"], "op": s["op"]}
        if "x_h" in s:
            d["x"] = dev(s["x_h"])
        if "binmode" in s:
            d["binmode"] = s["binmode"]
        spec.append(d)
    return mm.Batch(spec), spec


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_batch_matches_oracle(mm, ref, seed):
    series = mixed_series(seed, 60)
    b, spec = to_batch(mm, series)
    for graph in (False, True, True):
        b.out.fill_(-7)
        b.run(graph=graph)
        res = b.results()
        for i, s in enumerate(series):
            exp = oracle_result(ref, s)
            got = res[i].cpu().numpy()
            assert np.array_equal(got, exp), (seed, i, s["op"], len(s["y_h"]), s["n_out"], graph)
    b.close()


def test_graph_replay_sees_new_data(mm, ref):
    series = mixed_series(7, 20)
    b, spec = to_batch(mm, series)
    b.run(graph=True)
    r = np.random.default_rng(9)
    for s, d in zip(series, spec):
        s["y_h"] = (s["y_h"] * -1.5 + r.standard_normal(len(s["y_h"]))).astype(s["y_h"].dtype)
        d["y"].copy_(dev(s["y_h"]))
    b.run(graph=True)
    res = b.results()
    for i, s in enumerate(series):
        assert np.array_equal(res[i].cpu().numpy(), oracle_result(ref, s)), i
    b.close()


def test_batch_equals_single_calls(mm):
    lens, nouts = synth.batch_shapes(256, seed=3, lo=3.0, hi=6.0)
    series = [{"y": dev(synth.random_walk(int(n), seed=100 + i, dtype=np.float32)),
               "n_out": int(k), "r_ps": 4} for i, (n, k) in enumerate(zip(lens, nouts))]
    b = mm.Batch(series)
    b.run(graph=True)
    res = b.results()
    for i, s in enumerate(series):
        single = mm.minmaxlttb(s["y"], s["n_out"], 4)
        assert torch.equal(res[i], single), i
    b.close()


@pytest.mark.slow
def test_batched_4096_series(mm, ref):
    """4096 series, lengths round(10^U(3,7)), n_out in {200..4000}, r_ps = 4, float32
    random walks: every series equals a single-series call; a seeded sample of 96
    series (and the 8 longest) equals the oracle."""
    lens, nouts = synth.batch_shapes(4096, seed=0)
    ys = [synth.random_walk(int(n), seed=1000 + i, dtype=np.float32) for i, n in enumerate(lens)]
    series = [{"y": dev(y), "n_out": int(k), "r_ps": 4} for y, k in zip(ys, nouts)]
    b = mm.Batch(series)
    b.run(graph=True)
    res = b.results()
    pick = set(np.random.default_rng(1).choice(4096, 96, replace=False).tolist())
    pick |= set(np.argsort(lens)[-8:].tolist())
    for i in sorted(pick):
        assert np.array_equal(res[i].cpu().numpy(), ref.minmaxlttb(ys[i], int(nouts[i]), 4)), i
    for i, s in enumerate(series):
        assert torch.equal(res[i], mm.minmaxlttb(s["y"], s["n_out"], 4)), i
    b.close()
