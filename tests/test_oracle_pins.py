"""The oracle against its pins (CPU only): worked examples, numpy argmin/argmax,
exact rational LTTB, brute-force x-width bins, invariants and symmetries."""
import pytest

import pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(ref, check):
    check(ref)


def test_oracle_rejects_bad_arguments(ref):
    import numpy as np
    y = np.arange(10, dtype=np.float64)
    with pytest.raises(ValueError):
        ref.minmaxlttb(y, 2, 4)        # n_out < 3 with n_out < n
    with pytest.raises(ValueError):
        ref.minmaxlttb(y, 4, 1)        # r_ps < 2
    with pytest.raises(ValueError):
        ref.lttb(y, 2)
    with pytest.raises(ValueError):
        ref.minmax_preselect(y, 1, 1)  # B = 0
    with pytest.raises(ValueError):
        ref.minmax_preselect(y, 4, 2, binmode="xwidth")  # x-width bins need int64 x


def _lttb_variant(y, n_out, area, total):
    """LTTB on implicit x with a chosen area and sum rule, used only to show that the
    rounding fixtures G and H separate the rules they are meant to separate."""
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
            v = area(0.0 + a, y[a], float(b), y[b], xc, yc)
            if best is None or v > best:
                best, pick = v, b
        out.append(pick)
        a = pick
    return out + [m - 1]


def test_rounding_fixtures_separate_the_rules():
    """Cases G and H of the worked examples would change under the rounding a
    plausible mistake uses (a fused multiply-add, another summation order): the
    fixture itself, checked with Python's IEEE doubles and exact rationals."""
    import json
    from fractions import Fraction as F
    cases = {c["name"]: c for c in json.load(open(pins.GOLDEN))["cases"]}

    def rnd(q):
        return q.numerator / q.denominator  # correctly rounded int / int

    def separate(xa, ya, xb, yb, xc, yc):
        return abs((xa - xc) * (yb - ya) - (xa - xb) * (yc - ya))

    def fma_a(xa, ya, xb, yb, xc, yc):
        return abs(rnd(F(xa - xc) * F(yb - ya) - F((xa - xb) * (yc - ya))))

    def fma_b(xa, ya, xb, yb, xc, yc):
        return abs(rnd(F((xa - xc) * (yb - ya)) - F(xa - xb) * F(yc - ya)))

    def left_to_right(v):
        s = 0.0
        for e in v:
            s = s + e
        return s

    def right_to_left(v):
        return left_to_right(v[::-1])

    def exact(v):
        return rnd(sum(F(e) for e in v))

    g = cases["G_area_rounding_no_fma"]
    yg = [float.fromhex(h) for h in g["y_hex"]]
    assert _lttb_variant(yg, g["n_out"], separate, left_to_right) == g["expect"]
    for contracted in (fma_a, fma_b):
        assert _lttb_variant(yg, g["n_out"], contracted, left_to_right) == g["contracted_expect"]
    h = cases["H_mean_left_to_right"]
    yh = [float(v) for v in h["y"]]
    assert _lttb_variant(yh, h["n_out"], separate, left_to_right) == h["expect"]
    assert _lttb_variant(yh, h["n_out"], separate, right_to_left) == h["right_to_left_expect"]
    assert _lttb_variant(yh, h["n_out"], separate, exact) == h["exact_sum_expect"]


def test_rounding_cases_separate_the_rules(ref):
    """The larger constructions the GPU tests use (tests/rounding_cases.py) also
    change their pick under a fused multiply-add or another summation order, and
    the oracle takes the separately rounded, left-to-right pick on each."""
    import rounding_cases as rc
    for name, y, n_out in rc.area_cases():
        s = rc.pick_variant(y, n_out)
        assert rc.pick_variant(y, n_out, area="fma_first") != s, name
        assert rc.pick_variant(y, n_out, area="fma_second") != s, name
        assert ref.lttb(y, n_out).tolist() == s, name
    for name, y, n_out in rc.mean_cases():
        s = rc.pick_variant(y, n_out)
        assert rc.pick_variant(y, n_out, total="right_to_left") != s, name
        assert rc.pick_variant(y, n_out, total="exact") != s, name
        assert ref.lttb(y, n_out).tolist() == s, name
