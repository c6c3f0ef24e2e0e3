"""Failure detection on the GPU without a fault: every device-side wait of the
library is bounded.  A barrier that one CTA never reaches runs out after its 2 s
limit, the kernel records bit 1 in the workspace status word and returns, and the
context stays usable: the next call returns the oracle's indices."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["fused", "grid"])
def test_unsatisfied_barrier_times_out_and_reports(mm, ref, which):
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    kind = {"fused": mm.DIAG_FUSED_BARRIER, "grid": mm.DIAG_GRID_BARRIER}[which]
    mm.diag_wait_timeout(kind, ws)
    assert mm.workspace_status(ws) == 1  # bit 1: a bounded wait timed out
    y = synth.random_walk(100_000, seed=3, dtype=np.float32)
    got = mm.minmaxlttb(torch.from_numpy(y).cuda(), 500, 4).cpu().numpy()
    assert np.array_equal(got, ref.minmaxlttb(y, 500, 4))
