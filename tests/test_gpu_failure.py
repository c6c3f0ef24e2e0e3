"""Failure detection on the GPU without a fault: every device-side wait of the
library is bounded, and a device-side check reports violated preconditions.  A grid
barrier that one CTA never reaches, or a staged-stream mbarrier that no copy completes,
runs out after its 2 s limit, the kernel records bit 1 in the workspace status word and
returns, and the context stays usable: the next call returns the oracle's indices."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["fused", "grid", "mbarrier"])
def test_unsatisfied_barrier_times_out_and_reports(mm, ref, which):
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    kind = {"fused": mm.DIAG_FUSED_BARRIER, "grid": mm.DIAG_GRID_BARRIER, "mbarrier": mm.DIAG_MBARRIER}[which]
    mm.diag_wait_timeout(kind, ws)
    assert mm.workspace_status(ws) == 1  # bit 1: a bounded wait timed out
    y = synth.random_walk(100_000, seed=3, dtype=np.float32)
    got = mm.minmaxlttb(torch.from_numpy(y).cuda(), 500, 4).cpu().numpy()
    assert np.array_equal(got, ref.minmaxlttb(y, 500, 4))


def test_precondition_check(mm):
    r = np.random.default_rng(4)
    n = 1_000_003
    y = synth.random_walk(n, seed=4, dtype=np.float64)
    x = np.cumsum(r.integers(0, 5, n)).astype(np.int64)
    yd, xd = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    assert mm.check_series(yd) == set()
    assert mm.check_series(yd, xd) == set()
    assert mm.check_series(yd.float(), xd.double()) == set()
    bad = y.copy()
    bad[n - 1] = np.nan
    assert mm.check_series(torch.from_numpy(bad).cuda(), xd) == {"y_nan"}
    assert mm.check_series(torch.from_numpy(bad).float().cuda()) == {"y_nan"}
    xb = x.copy()
    xb[n // 2] = xb[n // 2 + 1] + 1  # one decrease
    assert mm.check_series(yd, torch.from_numpy(xb).cuda()) == {"x_decreases"}
    xf = x.astype(np.float64)
    xf[7] = np.inf
    assert mm.check_series(yd, torch.from_numpy(xf).cuda()) == {"x_nonfinite", "x_decreases"}
    assert mm.check_series(yd[:0]) == set()
