"""The GPU path keeps the oracle's roundings (readings R6: FP64 area with every
product and difference rounded on its own; R7: next-bucket mean summed left to
right, then one division).  Worked examples G and H, and the same constructions at
bucket sizes that reach every LTTB engine, run through each single-series launch
path and through a batch with and without a CUDA graph; each must equal the worked
example's hand-derived result where there is one and the oracle's everywhere."""
import json

import numpy as np
import pytest
import torch

import pins
import rounding_cases as rc

pytestmark = pytest.mark.gpu

PATHS = ["split", "fused_tail", "fused"]


def _cases():
    golden = {c["name"]: c for c in json.load(open(pins.GOLDEN))["cases"]}
    g = golden["G_area_rounding_no_fma"]
    h = golden["H_mean_left_to_right"]
    out = [("G", np.array([float.fromhex(v) for v in g["y_hex"]]), g["n_out"], g["expect"]),
           ("H", np.array(h["y"], np.float64), h["n_out"], h["expect"])]
    out += [(name, y, n_out, None) for name, y, n_out in rc.area_cases() + rc.mean_cases()]
    return out


CASES = _cases()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("path", PATHS)
def test_rounding_cases_every_path(mm, ref, path):
    mm.set_single_path({"split": mm.PATH_SPLIT, "fused_tail": mm.PATH_FUSED_TAIL,
                        "fused": mm.PATH_FUSED}[path])
    try:
        for name, y, n_out, expect in CASES:
            exp = ref.lttb(y, n_out)
            if expect is not None:
                assert exp.tolist() == expect, name
            yd = dev(y)
            got = mm.lttb(yd, n_out).cpu().numpy()
            assert np.array_equal(got, exp), (path, name, got, exp)
            # MinMaxLTTB with r_ps * n_out >= n is LTTB on every point (R15)
            r_ps = -(-len(y) // n_out)
            got = mm.minmaxlttb(yd, n_out, max(2, r_ps)).cpu().numpy()
            assert np.array_equal(got, exp), (path, name, "minmaxlttb", got, exp)
    finally:
        mm.set_single_path(mm.PATH_AUTO)


def test_rounding_cases_in_a_batch(mm, ref):
    spec = [{"y": dev(y), "n_out": n_out, "op": "lttb"} for _, y, n_out, _ in CASES]
    b = mm.Batch(spec)
    for graph in (False, True, True):
        b.out.fill_(-1)
        b.run(graph=graph)
        res = b.results()
        for (name, y, n_out, _), r in zip(CASES, res):
            assert np.array_equal(r.cpu().numpy(), ref.lttb(y, n_out)), (name, graph)
    b.close()
