"""Zoom-window server (continuous batching): every result equals the single-series
call on the window (and the oracle on a sample), results are the same alone and in
the mix, and malformed / oversize requests and a full queue are refused on the host."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def resident():
    ys = {
        "walk32": synth.random_walk(2_000_000, seed=11, dtype=np.float32),
        "walk64": synth.random_walk(1_000_000, seed=12, dtype=np.float64),
        "ties32": np.random.default_rng(13).integers(-3, 4, 500_000).astype(np.float32),
    }
    x64 = synth.exp_gaps_x(1_000_000, seed=12, mean_gap=20.0, big_gaps=4, big_gap=100_000)
    dev = {k: torch.from_numpy(v).cuda() for k, v in ys.items()}
    return ys, x64, dev, torch.from_numpy(x64).cuda()


def make_requests(seed, count, sizes, x_series):
    r = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        s = int(r.integers(0, len(sizes)))
        n = sizes[s]
        width = int(np.clip(np.rint(10 ** r.uniform(1, np.log10(n))), 3, n))
        start = int(r.integers(0, n - width + 1))
        n_out = int(r.choice([3, 4, 17, 200, 1000, 4000]))
        r_ps = int(r.choice([2, 4, 8]))
        bm = 1 if (s == x_series and r.random() < 0.6) else 0
        reqs.append((s, start, start + width, n_out, r_ps, bm))
    return reqs


def start_server(mm, resident, **kw):
    ys, x64, dev, xd = resident
    srv = mm.Server(**kw)
    ids = [srv.add_series(dev["walk32"]), srv.add_series(dev["walk64"], xd), srv.add_series(dev["ties32"])]
    return srv, ids


def single(mm, resident, q):
    ys, x64, dev, xd = resident
    key = ["walk32", "walk64", "ties32"][q[0]]
    y = dev[key][q[1]:q[2]]
    x = xd[q[1]:q[2]] if key == "walk64" else None
    return mm.minmaxlttb(y, q[3], q[4], x=x, binmode=q[5]).cpu().numpy() + q[1]


def test_server_results_match_single_calls_and_oracle(mm, ref, resident):
    ys, x64, dev, xd = resident
    srv, sids = start_server(mm, resident, streams=3, max_batch=64, workspace_bytes_per_stream=128 << 20)
    reqs = make_requests(0, 300, [2_000_000, 1_000_000, 500_000], 1)
    ids = [srv.submit(*q) for q in reqs]
    res = [srv.wait(i)[0] for i in ids]
    for q, got in zip(reqs, res):
        assert np.array_equal(got, single(mm, resident, q)), q
    keys = ["walk32", "walk64", "ties32"]
    for k in range(0, 300, 10):
        q = reqs[k]
        y = ys[keys[q[0]]][q[1]:q[2]]
        x = x64[q[1]:q[2]] if q[0] == 1 else None
        exp = ref.minmaxlttb(y, q[3], q[4], x=x, binmode=["index", "xwidth"][q[5]]) + q[1]
        assert np.array_equal(res[k], exp), q
    st = srv.stats()
    assert st["completed"] == 300 and st["batches"] >= 1
    srv.close()


def test_alone_equals_in_mix(mm, resident):
    reqs = make_requests(1, 120, [2_000_000, 1_000_000, 500_000], 1)
    alone_srv, _ = start_server(mm, resident, streams=1, max_batch=1, workspace_bytes_per_stream=64 << 20)
    alone = [alone_srv.wait(alone_srv.submit(*q))[0] for q in reqs]
    alone_srv.close()
    mix_srv, _ = start_server(mm, resident, streams=2, max_batch=32, workspace_bytes_per_stream=128 << 20)
    ids = [mix_srv.submit(*q) for q in reqs]
    mixed = [mix_srv.wait(i)[0] for i in ids]
    st = mix_srv.stats()
    mix_srv.close()
    for a, b in zip(alone, mixed):
        assert np.array_equal(a, b)
    assert st["mean_batch"] > 1.0  # requests really were batched together


def test_replay_trace(mm, resident):
    srv, _ = start_server(mm, resident, streams=2, max_batch=128, workspace_bytes_per_stream=128 << 20)
    reqs = make_requests(2, 400, [2_000_000, 1_000_000, 500_000], 1)
    offs = np.cumsum(np.random.default_rng(3).exponential(1.0 / 4000.0, len(reqs))).tolist()
    qs = [mm.Request(*q) for q in reqs]
    ids, st = srv.replay(qs, offs)
    assert all(s == 0 for s in st)
    srv.drain()
    stats = srv.stats()
    assert stats["completed"] == 400
    assert 0 < stats["latency_p50_s"] <= stats["latency_p99_s"] <= stats["latency_max_s"] < 5.0
    for q, i in zip(reqs[:40], ids[:40]):
        assert np.array_equal(srv.wait(i)[0], single(mm, resident, q))
    srv.close()


def test_malformed_oversize_and_full_queue(mm, resident):
    srv, _ = start_server(mm, resident, streams=1, max_batch=4, max_pending=3,
                          workspace_bytes_per_stream=4 << 20)
    bad = [(7, 0, 10, 5, 4, 0),          # unknown series
           (0, 10, 10, 5, 4, 0),         # empty window
           (0, -1, 10, 5, 4, 0),         # negative start
           (0, 0, 2_000_001, 5, 4, 0),   # past the end
           (0, 0, 1000, 2, 4, 0),        # n_out < 3
           (0, 0, 1000, 5000, 4, 0),     # n_out > max_n_out
           (0, 0, 1000, 50, 1, 0),       # r_ps < 2
           (0, 0, 1000, 50, 4, 1)]       # x-width bins on a series without x
    for q in bad:
        with pytest.raises(mm.MMLTTBError) as e:
            srv.submit(*q)
        assert e.value.code == mm.EINVAL, q
    with pytest.raises(mm.MMLTTBError) as e:  # 4000*64/2 bins: workspace beyond 4 MiB
        srv.submit(0, 0, 2_000_000, 4000, 64, 0)
    assert e.value.code == mm.ENOSPC
    codes = []
    ids = []
    for k in range(200):  # flood a 3-deep queue: some submissions must bounce
        try:
            ids.append(srv.submit(0, 0, 1_000_000, 100, 4, 0))
        except mm.MMLTTBError as err:
            codes.append(err.code)
    assert codes and all(c == mm.EBUSY for c in codes)
    srv.drain()
    for i in ids:
        assert len(srv.wait(i)[0]) == 100
    srv.close()


def test_batches_overlap_on_the_device(mm, resident):
    """Continuous batching, not a queue: under a burst, batches are admitted while
    other batches of the same server are still in flight on the device (the
    server counts them at admission), and results stay those of single calls.  A
    one-slot server never overlaps, so the count is not trivially positive."""
    reqs = make_requests(4, 240, [2_000_000, 1_000_000, 500_000], 1)
    srv, _ = start_server(mm, resident, streams=3, max_batch=8, workspace_bytes_per_stream=128 << 20)
    ids = [srv.submit(*q) for q in reqs]  # a burst: the queue fills faster than slots free up
    res = [srv.wait(i)[0] for i in ids]
    st = srv.stats()
    srv.close()
    assert st["batches"] >= 240 // 8
    assert st["overlapped_batches"] > 0
    assert 2 <= st["max_batches_in_flight"] <= 3
    for q, got in zip(reqs[::8], res[::8]):
        assert np.array_equal(got, single(mm, resident, q)), q
    one, _ = start_server(mm, resident, streams=1, max_batch=8, workspace_bytes_per_stream=128 << 20)
    ids = [one.submit(*q) for q in reqs[:64]]
    for i in ids:
        one.wait(i)
    st1 = one.stats()
    one.close()
    assert st1["overlapped_batches"] == 0 and st1["max_batches_in_flight"] == 1
