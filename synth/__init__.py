"""Seeded synthetic time series shaped like the MinMaxLTTB workloads.

The paper evaluates on templates of an earlier study that are not available here;
these seeded series stand in for them.  This module holds none of the method's
arithmetic (no bins, extrema, areas or means): only random numbers, walks, sines,
spikes and gaps.  The tests feed the same bytes to the oracle and to the GPU path.

Every generator is deterministic in (seed, n) and independent of the number of
threads: the series is cut into chunks of 2**22 points, chunk k draws from its own
PCG64 stream SeedSequence(seed, spawn_key=(tag, k)), and walks are accumulated in
FP64 chunk by chunk (chunk-local cumulative sums plus the running end value of the
previous chunks).  Values of sin() may differ in the last bit between host
architectures, so comparisons are always made on the bytes of one machine.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 1 << 22
TAG_STEPS, TAG_GAPS, TAG_SPIKE, TAG_SIGN, TAG_BIG, TAG_BATCH = 1, 2, 3, 4, 5, 6


def _rng(seed, tag, k=0):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(entropy=seed, spawn_key=(tag, k))))


def _chunks(n):
    return [(a, min(a + CHUNK, n)) for a in range(0, n, CHUNK)]


def _workers():
    return max(1, min(32, os.cpu_count() or 1))


def _map(fn, items):
    if len(items) <= 1:
        return [fn(it) for it in items]
    with ThreadPoolExecutor(_workers()) as ex:
        return list(ex.map(fn, items))


def _steps(seed, sigma, k, m):
    s = _rng(seed, TAG_STEPS, k).standard_normal(m)
    if sigma != 1.0:
        s *= sigma
    return s


def random_walk(n, seed=0, dtype=np.float32, sigma=1.0, out=None, extra=None):
    """Gaussian random walk y[i] = sum_{k<=i} s_k, s_k ~ N(0, sigma^2), FP64, stored as dtype.

    extra(a, b, v) may add further FP64 terms to the chunk v = y[a:b] before rounding.
    Each chunk's steps are drawn once: the chunk-local FP64 cumulative sums are kept
    (in `out` itself for float64 output, else in a temporary float64 array) until the
    offsets of the chunks before them are known."""
    n = int(n)
    if out is None:
        out = np.empty(n, dtype=dtype)
    if n == 0:
        return out
    chunks = _chunks(n)
    tmp = out if out.dtype == np.float64 else np.empty(n, np.float64)

    def local(k_ab):
        k, (a, b) = k_ab
        np.cumsum(_steps(seed, sigma, k, b - a), out=tmp[a:b])
        return tmp[b - 1]
    ends = _map(local, list(enumerate(chunks)))
    offs = [0.0]
    for e in ends[:-1]:
        offs.append(offs[-1] + e)  # sequential FP64

    def fill(k_ab):
        k, (a, b) = k_ab
        v = tmp[a:b]
        v += offs[k]
        if extra is not None:
            extra(a, b, v)
        if tmp is not out:
            out[a:b] = v
    _map(fill, list(enumerate(chunks)))
    return out


def random_walks(lengths, seed0, dtype=np.float32):
    """Independent walks random_walk(lengths[i], seed=seed0 + i), generated on a pool
    of threads (many short series, each a single chunk)."""
    return _map(lambda i_n: random_walk(int(i_n[1]), seed=seed0 + i_n[0], dtype=dtype),
                list(enumerate(lengths)))


def walk_sines_spikes(n, seed=0, dtype=np.float32, periods=(1e3, 1e5, 1e7), spike_p=1e-4,
                      spike_sigma=50.0, out=None):
    """Random walk (sigma 1) + sines of the given periods with amplitude sqrt(period)
    (the walk's spread over one period) + spikes of +-spike_sigma with probability
    spike_p per point."""
    def extra(a, b, v):
        i = np.arange(a, b, dtype=np.float64)
        for p in periods:
            v += np.sqrt(p) * np.sin((2.0 * np.pi / p) * i)
        k = a // CHUNK
        hit = _rng(seed, TAG_SPIKE, k).random(b - a) < spike_p
        if hit.any():
            sign = np.where(_rng(seed, TAG_SIGN, k).random(b - a) < 0.5, -1.0, 1.0)
            v += np.where(hit, spike_sigma * sign, 0.0)
    return random_walk(n, seed, dtype, 1.0, out, extra)


def exp_gaps_x(n, seed=0, mean_gap=1000.0, big_gaps=5, big_gap=1_000_000_000, out=None):
    """Strictly increasing int64 x: x[0] = 0, x[i] = x[i-1] + g_i with
    g_i = max(1, round(Exp(mean_gap))), except big_gaps seeded positions where
    g_i = big_gap."""
    n = int(n)
    if out is None:
        out = np.empty(n, dtype=np.int64)
    if n == 0:
        return out
    chunks = _chunks(n)
    big = np.sort(_rng(seed, TAG_BIG).choice(np.arange(1, n), size=min(big_gaps, n - 1), replace=False)) \
        if n > 1 and big_gaps > 0 else np.empty(0, np.int64)

    def gaps(k, a, b):
        g = np.rint(_rng(seed, TAG_GAPS, k).exponential(mean_gap, b - a))
        g = np.maximum(g, 1.0).astype(np.int64)
        if a == 0:
            g[0] = 0
        sel = big[(big >= a) & (big < b)]
        g[sel - a] = big_gap
        return g

    def total(k_ab):
        k, (a, b) = k_ab
        return int(gaps(k, a, b).sum())
    tot = _map(total, list(enumerate(chunks)))
    offs = np.concatenate([[0], np.cumsum(tot)[:-1]]).astype(np.int64)

    def fill(k_ab):
        k, (a, b) = k_ab
        np.cumsum(gaps(k, a, b), out=out[a:b])
        out[a:b] += offs[k]
    _map(fill, list(enumerate(chunks)))
    return out


def ties_series(n, seed=0, levels=5, dtype=np.float32):
    """Small-integer values in [-levels, levels]: many exact ties, exact arithmetic."""
    return _rng(seed, 11).integers(-levels, levels + 1, size=int(n)).astype(dtype)


def signed_zero_series(n, seed=0, dtype=np.float32):
    """Values drawn from {-0.0, +0.0, -1, +1}: exercises the -0.0 == +0.0 ties."""
    v = np.array([-0.0, 0.0, -1.0, 1.0], dtype=dtype)
    return v[_rng(seed, 12).integers(0, 4, size=int(n))]


def batch_shapes(n_series=4096, seed=0, lo=3.0, hi=7.0, nout_lo=200, nout_hi=4000):
    """Lengths round(10**U(lo, hi)) and n_out uniform in {nout_lo..nout_hi}."""
    r = _rng(seed, TAG_BATCH)
    lens = np.rint(10.0 ** r.uniform(lo, hi, n_series)).astype(np.int64)
    nouts = r.integers(nout_lo, nout_hi + 1, n_series).astype(np.int64)
    return lens, nouts
