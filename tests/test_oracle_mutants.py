"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that at
least one pin catches each: the pins are strong enough to trust the oracle."""
import json
import os
import platform
import subprocess
import sys
import tempfile

import pytest

import pins
from oracle import CFLAGS, SRC, Oracle

# (name, original text, mutated text); each original must occur exactly once.
MUTANTS = [
    ("area_sign_first_term", "(xa - xc) * (yb - ya)", "(xa - xc) * (ya - yb)"),
    ("area_wrong_point", "(xa - xb) * (yc - ya)", "(xa - xb) * (yc - yb)"),
    ("area_transposed_operand", "(xa - xb) * (yc - ya)", "(xb - xa) * (yc - ya)"),
    ("area_dropped_term", "fabs((xa - xc) * (yb - ya) - (xa - xb) * (yc - ya))", "fabs((xa - xc) * (yb - ya))"),
    ("mean_count_off_by_one", "double cnt = (double)(nhi - nlo);", "double cnt = (double)(nhi - nlo + 1);"),
    ("mean_uses_x_for_y", "sy = sy + y_at(y, ydt, IDX(p));", "sy = sy + x_at(x, xk, IDX(p));"),
    ("next_bucket_is_current", "if (j + 1 < K) { nlo = hi; nhi = part_start(j + 2, N, K); }",
     "if (j + 1 < K) { nlo = lo; nhi = hi; }"),
    # R6: one fused multiply-add in place of the separately rounded products, either way round
    ("area_fma_second_product_rounded", "double area = fabs((xa - xc) * (yb - ya) - (xa - xb) * (yc - ya));",
     "double area = fabs(fma(xa - xc, yb - ya, -((xa - xb) * (yc - ya))));"),
    ("area_fma_first_product_rounded", "double area = fabs((xa - xc) * (yb - ya) - (xa - xb) * (yc - ya));",
     "double area = fabs(fma(-(xa - xb), yc - ya, (xa - xc) * (yb - ya)));"),
    # R7: the next bucket summed in another order, or compensated
    ("mean_right_to_left", "for (int64_t p = nlo; p < nhi; p++) {\n            sx = sx + x_at(x, xk, IDX(p));",
     "for (int64_t p = nhi - 1; p >= nlo; p--) {\n            sx = sx + x_at(x, xk, IDX(p));"),
    ("mean_compensated_sum",  # Neumaier's compensated sum: exact on most buckets
     "double sx = 0.0, sy = 0.0;\n        for (int64_t p = nlo; p < nhi; p++) {\n            sx = sx + x_at(x, xk, IDX(p));\n"
     "            sy = sy + y_at(y, ydt, IDX(p));\n        }\n        double cnt = (double)(nhi - nlo);\n"
     "        double xc = sx / cnt, yc = sy / cnt;",
     "double sx = 0.0, sy = 0.0, comp = 0.0;\n        for (int64_t p = nlo; p < nhi; p++) {\n"
     "            sx = sx + x_at(x, xk, IDX(p));\n"
     "            double v = y_at(y, ydt, IDX(p)), t = sy + v;\n"
     "            comp += fabs(sy) >= fabs(v) ? (sy - t) + v : (v - t) + sy;\n            sy = t;\n        }\n"
     "        double cnt = (double)(nhi - nlo);\n        double xc = sx / cnt, yc = (sy + comp) / cnt;"),
    ("lttb_tie_last_wins", "if (p == lo || area > best)", "if (p == lo || area >= best)"),
    ("previous_pick_not_advanced", "        a = pick;\n", "\n"),
    ("bucket_start_ceil", "return (int64_t)(num / (uint64_t)c) + 1;",
     "return (int64_t)((num + (uint64_t)c - 1) / (uint64_t)c) + 1;"),
    ("minmax_tie_last_min", "(R8, R10) */\n            if (v < vmin[b])", "(R8, R10) */\n            if (v <= vmin[b])"),
    ("minmax_tie_last_max", "(R8, R10) */\n            if (v < vmin[b]) { vmin[b] = v; imin[b] = p; }\n            if (v > vmax[b])",
     "(R8, R10) */\n            if (v < vmin[b]) { vmin[b] = v; imin[b] = p; }\n            if (v >= vmax[b])"),
    ("m4_tie_last_min", "            } else {\n                if (v < vmin[b])", "            } else {\n                if (v <= vmin[b])"),
    ("minmax_includes_first_point", "for (int64_t p = 1; p <= n - 2; p++) {", "for (int64_t p = 0; p <= n - 2; p++) {"),
    ("minmax_includes_last_point", "for (int64_t p = 1; p <= n - 2; p++) {", "for (int64_t p = 1; p <= n - 1; p++) {"),
    ("last_point_dropped", "    out[m++] = n - 1;\n", "\n"),
    ("no_dedupe_equal_extrema", "if (hi != lo) out[m++] = hi;", "out[m++] = hi;"),
    ("bin_edge_strict", "while (!fx && next <= here) {\n            b++;\n            next = NEXT_BOUND(b);",
     "while (!fx && next < here) {\n            b++;\n            next = NEXT_BOUND(b);"),
    ("m4_bin_edge_strict", "while (!fx && next <= here) {\n            b++;\n            next = NEXT_BOUND4(b);",
     "while (!fx && next < here) {\n            b++;\n            next = NEXT_BOUND4(b);"),
    ("f64x_edge_strict", "while (nextf <= xf[p]) {\n                b++;\n                nextf = NEXT_EDGE_F(b);",
     "while (nextf < xf[p]) {\n                b++;\n                nextf = NEXT_EDGE_F(b);"),
    ("f64x_edge_formula", "#define NEXT_EDGE_F(bb) ((bb) + 1 >= B ? INFINITY : xf0 + ((double)((bb) + 1) * Df) / (double)B)",
     "#define NEXT_EDGE_F(bb) ((bb) + 1 >= B ? INFINITY : xf0 + ((double)(bb) * Df) / (double)B)"),
    ("bins_from_r_ps_not_halved", "int64_t B = n_out * (int64_t)r_ps / 2;\n    if (B < 1) return MMO_EINVAL;",
     "int64_t B = n_out * (int64_t)r_ps;\n    if (B < 1) return MMO_EINVAL;"),
    ("m4_last_not_updated", "            last[b] = p;\n", "\n"),
    ("m4_bins_over_interior", "    for (int64_t p = 0; p < n; p++) {\n        if (fx) {\n            while (nextf <= xf[p]) {\n                b++;\n                nextf = NEXT_EDGE_F4(b);",
     "    for (int64_t p = 1; p < n; p++) {\n        if (fx) {\n            while (nextf <= xf[p]) {\n                b++;\n                nextf = NEXT_EDGE_F4(b);"),
    ("nan_last_wins", "        } else if (nan_aware && hasnan[b]) {\n            /* the bin's first NaN decides both extremes (R18) */\n        } else if (nan_aware && isnan(v)) {",
     "        } else if (nan_aware && isnan(v)) {"),
    ("nan_ignored", "            hasnan[b] = 1; imin[b] = p; imax[b] = p;\n        } else {\n            /* strict",
     "            hasnan[b] = 0;\n        } else {\n            /* strict"),
    ("no_lttb_when_rps_covers_n", "if ((int64_t)r_ps * n_out >= n) return mmo_lttb(y, ydt, x, xk, n, n_out, out);", ""),
    ("raster_sample_offset", "(0.25f * (float)i + 0.125f)", "(0.25f * (float)i)"),
    ("raster_strict_width", "return d2 <= 1.0f;", "return d2 < 1.0f;"),
    ("raster_no_row_flip", "double t = flip ? (b - v) : (v - a);", "double t = (v - a);"),
    ("raster_no_bbox_margin", "double c0 = floor((double)lox - 1.0), c1 = floor((double)hix + 1.0);",
     "double c0 = floor((double)lox), c1 = floor((double)hix);"),
    ("raster_no_clamp", "if (t > 1.0f) t = 1.0f;", ""),
    ("raster_intensity_floor", "out[p] = (uint8_t)((inked * 255 + 8) / 16);", "out[p] = (uint8_t)((inked * 255) / 16);"),
    ("pem_margin_inclusive", "if (d > margin) over++;", "if (d >= margin) over++;"),
    ("mask_no_dilation", "for (int rr = r - 1; rr <= r + 1 && !inmask; rr++)", "for (int rr = r; rr <= r && !inmask; rr++)"),
]


def _build_mutant(tmpdir, name, old, new, cflags=CFLAGS):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {name}: anchor text found {src.count(old)} times"
    path_c = os.path.join(tmpdir, f"{name}.c")
    path_so = os.path.join(tmpdir, f"lib{name}.so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", *cflags, path_c, "-o", path_so, "-lm"], check=True)
    return path_so


@pytest.fixture(scope="module")
def tmpdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


_CHILD = r"""
import json, sys
sys.path[:0] = [sys.argv[2], sys.argv[3]]
import pins
from oracle import Oracle
o = Oracle(sys.argv[1])
caught = []
for check in pins.ALL_CHECKS:
    try:
        check(o)
    except Exception as e:
        caught.append(check.__name__)
print(json.dumps(caught))
"""


def _caught(so):
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, "-c", _CHILD, so, here, os.path.dirname(here)],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return ["<crashed>"]
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_has_fma():
    if platform.machine() in ("aarch64", "arm64"):
        return True  # every AArch64 core has FMADD
    try:
        return " fma " in open("/proc/cpuinfo").read().replace("\n", " ")
    except OSError:
        return False


@pytest.mark.skipif(not _cpu_has_fma(), reason="this CPU has no FMA instruction to contract into")
def test_contracting_build_is_caught(tmpdir):
    """The unmodified oracle compiled the way a careless build would be: GCC's
    default contraction (fused multiply-add wherever a product feeds a sum), with
    FMA instructions available.  Reading R6 forbids it; the pins must notice."""
    flags = [f for f in CFLAGS if f != "-ffp-contract=off"] + ["-ffp-contract=fast"]
    if platform.machine() == "x86_64":
        flags.append("-mfma")
    so = _build_mutant(tmpdir, "contracting_build", "double area", "double area", cflags=flags)
    assert "check_worked_examples" in _caught(so)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmpdir, name, old, new):
    # A child process: a mutant that writes out of bounds may crash, which also
    # counts as detected.
    so = _build_mutant(tmpdir, name, old, new)
    assert _caught(so), f"no pin detects the planted mistake {name}"
