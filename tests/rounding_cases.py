"""Inputs on which LTTB's pick depends on how the area and the next-bucket mean are
rounded (readings R6 and R7), at several bucket sizes, so that every LTTB engine
(small buckets, transition tables, the grid-wide argmax of big buckets) meets them.

  area_cases():  n_out = 3, one bucket; two candidates whose separately rounded FP64
                 areas tie (lowest index wins), while a fused multiply-add either
                 way round, or the exact area, makes the later one larger.
  mean_cases():  n_out = 4, two buckets of L points; the next bucket starts
                 1e16, 1, -1e16, 1, so its left-to-right FP64 sum is 1, right to
                 left or pairwise it is 0, and exactly it is 2; three candidates of
                 the first bucket each win under one of those sums.

Only inputs are built here (seeded, deterministic); expected results come from the
oracle.  pick_variant() restates the pick under another rounding rule so a CPU test
can show that each case separates the rules."""
import math
import random
from fractions import Fraction as F

import numpy as np


def _rnd(q):
    return q.numerator / q.denominator  # int / int is correctly rounded


def area_rule(name):
    def separate(xa, ya, xb, yb, xc, yc):
        return abs((xa - xc) * (yb - ya) - (xa - xb) * (yc - ya))

    def fma_first(xa, ya, xb, yb, xc, yc):   # fma(xa-xc, yb-ya, -(xa-xb)(yc-ya))
        return abs(_rnd(F(xa - xc) * F(yb - ya) - F((xa - xb) * (yc - ya))))

    def fma_second(xa, ya, xb, yb, xc, yc):  # fma(-(xa-xb), yc-ya, (xa-xc)(yb-ya))
        return abs(_rnd(F((xa - xc) * (yb - ya)) - F(xa - xb) * F(yc - ya)))
    return {"separate": separate, "fma_first": fma_first, "fma_second": fma_second}[name]


def sum_rule(name):
    def left_to_right(v):
        s = 0.0
        for e in v:
            s = s + e
        return s
    return {"left_to_right": left_to_right,
            "right_to_left": lambda v: left_to_right(list(v)[::-1]),
            "exact": lambda v: _rnd(sum(F(float(e)) for e in v))}[name]


def pick_variant(y, n_out, area="separate", total="left_to_right"):
    """LTTB (implicit x, bucket layout R1, next bucket of the last bucket R5) under
    the given area and sum rules."""
    area, total = area_rule(area), sum_rule(total)
    y = [float(v) for v in y]
    m, K = len(y), n_out - 2
    N = m - 2
    start = [j * N // K + 1 for j in range(K + 1)]
    out, a = [0], 0
    for j in range(K):
        nxt = range(start[j + 1], start[j + 2]) if j + 1 < K else range(m - 1, m)
        xc = total([float(p) for p in nxt]) / len(nxt)
        yc = total([y[p] for p in nxt]) / len(nxt)
        best, pick = None, None
        for b in range(start[j], start[j + 1]):
            v = area(float(a), y[a], float(b), y[b], xc, yc)
            if best is None or v > best:
                best, pick = v, b
        out.append(pick)
        a = pick
    return out + [m - 1]


def _area_case(m, seed):
    r = random.Random(seed)
    while True:
        ym = r.uniform(0.5, 2.0)
        y = [0.0] + [ym * b / (m - 1) * 0.999 for b in range(1, m - 1)] + [ym]
        i, j = sorted(r.sample(range(3, m - 1), 2))
        y[i] = r.uniform(2.0, 4.0)
        yj = (j * ym + abs(-(m - 1) * y[i] + i * ym)) / (m - 1)
        for k in range(-6, 7):
            v = yj
            for _ in range(abs(k)):
                v = math.nextafter(v, math.inf if k > 0 else -math.inf)
            yy = list(y)
            yy[j] = v
            s = pick_variant(yy, 3)
            if all(pick_variant(yy, 3, area=a) != s for a in ("fma_first", "fma_second")):
                return np.array(yy, np.float64)


def area_cases():
    """(name, y float64, n_out) with one bucket of 4, 38 and 98 candidates."""
    return [(f"area_m{m}", _area_case(m, 11 + m), 3) for m in (6, 40, 100)]


def mean_cases():
    """(name, y float64, n_out) with buckets of L = 4, 16 and 64 points."""
    out = []
    for L in (4, 16, 64):
        m = 2 * L + 2
        X = (3 * L + 1) / 2.0           # mean x of the next bucket (positions L+1..2L)
        c = -(-3 * L // 4)              # the third candidate's x
        u = 2.0
        s = u + 0.5 * (L - 1) / L / X   # wins at yc = 0
        t = u - 1.5 * (1 + c) / L / X   # wins at yc = 2/L
        y = np.zeros(m)
        y[1], y[L], y[c] = u, s, -t     # wins at yc = 1/L (left to right) at position 1
        y[L + 1:L + 5] = [1e16, 1.0, -1e16, 1.0]
        y[m - 1] = 1e16
        out.append((f"mean_L{L}", y, 4))
    return out
