"""The seeded generators: deterministic, chunk-stable, shaped as documented."""
import numpy as np

import synth


def test_walk_is_deterministic_and_chunk_stable():
    a = synth.random_walk(synth.CHUNK + 1234, seed=3, dtype=np.float64)
    b = synth.random_walk(synth.CHUNK + 1234, seed=3, dtype=np.float64)
    assert np.array_equal(a, b)
    c = synth.random_walk(1000, seed=3, dtype=np.float64)
    assert np.array_equal(a[:1000], c)  # a prefix is the same walk
    assert not np.array_equal(c, synth.random_walk(1000, seed=4, dtype=np.float64))
    steps = np.diff(a)
    assert abs(steps.std() - 1.0) < 0.01 and abs(steps.mean()) < 0.01


def test_float32_walk_rounds_the_float64_walk():
    a = synth.random_walk(50_000, seed=0, dtype=np.float64)
    b = synth.random_walk(50_000, seed=0, dtype=np.float32)
    assert np.array_equal(a.astype(np.float32), b)


def test_exp_gaps_x_strictly_increasing_with_big_gaps():
    x = synth.exp_gaps_x(200_000, seed=1, mean_gap=1000.0, big_gaps=5, big_gap=10**9)
    g = np.diff(x)
    assert x[0] == 0 and np.all(g >= 1)
    assert np.sum(g == 10**9) == 5
    small = g[g < 10**9]
    assert abs(small.mean() - 1000.0) < 20.0


def test_walk_sines_spikes_shape():
    y = synth.walk_sines_spikes(300_000, seed=2)
    assert y.dtype == np.float32 and len(y) == 300_000
    d = np.abs(np.diff(y.astype(np.float64)))
    assert np.sum(d > 40) > 10  # spikes of +-50 sigma occur at ~1e-4 per point


def test_batch_shapes():
    lens, nouts = synth.batch_shapes(4096, seed=0)
    assert lens.min() >= 1000 and lens.max() <= 10**7
    assert nouts.min() >= 200 and nouts.max() <= 4000
    assert 3.5e9 < lens.sum() < 5.5e9
