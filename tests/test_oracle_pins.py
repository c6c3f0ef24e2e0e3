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
