"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle's C source into a temporary directory, plants one
mistake (a dropped term, a wrong sign, a flipped comparison, an off-by-one),
compiles it, and runs the pin suite against that build in a child process.
The suite must fail on every mutant and pass on the unmodified copy.
"""
import os
import subprocess
import sys

import pytest

from oracle.oracle import compile_c

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ghn_oracle.c")

# (name, text to find, replacement); each find string occurs exactly once.
# Mutants that cannot change any result are left out: truncation instead of
# floor for training points (their quotient is never negative), and starting
# the walk at layer 0 instead of the first layer that reaches the box (the
# skipped layers are empty, so the buffer and the stop test are unchanged).
MUTANTS = [
    ("trunc_instead_of_floor_query", "float t = floorf((q[j] - g->origin[j]) / g->w[j]);",
     "float t = truncf((q[j] - g->origin[j]) / g->w[j]);"),
    ("origin_sign", "float t = (p[j] - g->origin[j]) / g->w[j];",
     "float t = (p[j] + g->origin[j]) / g->w[j];"),
    ("double_precision_key", "float t = (p[j] - g->origin[j]) / g->w[j];\n        c[j] = (int64_t)floorf(t);",
     "double t = ((double)p[j] - (double)g->origin[j]) / (double)g->w[j];\n        c[j] = (int64_t)floor(t);"),
    ("width_of_first_dimension", "float t = (p[j] - g->origin[j]) / g->w[j];",
     "float t = (p[j] - g->origin[j]) / g->w[0];"),
    ("no_split_clamp", "if (g->split[j] > 0 && c[j] > g->split[j] - 1) c[j] = g->split[j] - 1;",
     "(void)0;"),
    ("measure_misses_top", "int64_t s = u < GHN_ORACLE_MAX_SPLITS ? u : GHN_ORACLE_MAX_SPLITS;",
     "int64_t s = (u < GHN_ORACLE_MAX_SPLITS ? u : GHN_ORACLE_MAX_SPLITS) - 1;"),
    ("measure_skip_allowed", "if (c - prev > 1) ok = 0;", "if (c - prev > 2) ok = 0;"),
    ("measure_no_last_split_clamp", "if (!(t < (float)s)) return s - 1;",
     "if (!(t < (float)s + 1.0f)) return s;"),
    ("certified_edge_off_by_one", "double cu = (double)(c0[j] + L + 1);",
     "double cu = (double)(c0[j] + L + 2);"),
    ("certified_ignores_box", "if (c0[j] + L < g->cmax[j]) {", "if (1) {"),
    ("certified_without_full_buffer", "if (stop_rule == 2 && x.size == k && certified(",
     "if (stop_rule == 2 && certified("),
    ("origin_is_max", "if (points[i * d + j] < lo) lo = points[i * d + j];",
     "if (points[i * d + j] > lo) lo = points[i * d + j];"),
    ("dropped_distance_term", "acc = acc + s;", "acc = s;"),
    ("distance_index", "float t = q[j] - p[j];", "float t = q[0] - p[j];"),
    ("fused_distance", "float s = t * t;\n        acc = acc + s;", "acc = fmaf(t, t, acc);"),
    ("order_flipped", "return da < db || (da == db && ia < ib);",
     "return da > db || (da == db && ia < ib);"),
    ("tie_break_flipped", "return da < db || (da == db && ia < ib);",
     "return da < db || (da == db && ia > ib);"),
    ("stop_without_full_buffer", "if (stop_rule == 1 && x.size == k && !x.updated) break;",
     "if (stop_rule == 1 && !x.updated) break;"),
    ("stop_after_update", "if (stop_rule == 1 && x.size == k && !x.updated) break;",
     "if (stop_rule == 1 && x.size == k) break;"),
    ("shell_includes_inside", "if (cheb == L) {", "if (cheb <= L) {"),
    ("covers_off_by_one", "if (c0[j] - L > 0 || c0[j] + L < g->cmax[j]) covers = 0;",
     "if (c0[j] - L > 1 || c0[j] + L < g->cmax[j]) covers = 0;"),
    ("vote_tie_largest", "if (cnt > bestc || (cnt == bestc && lab < best)) {",
     "if (cnt > bestc || (cnt == bestc && lab > best)) {"),
    ("mean_over_k", "*(float*)pred = x.size ? (float)(sum / (double)x.size) : NAN;",
     "*(float*)pred = x.size ? (float)(sum / (double)k) : NAN;"),
    ("mean_in_single", "sum += (double)y;", "sum = (float)(sum + y);"),
    ("clamp_sign", "if (t > GHN_ORACLE_QCLAMP) t = GHN_ORACLE_QCLAMP;",
     "if (t > GHN_ORACLE_QCLAMP) t = -GHN_ORACLE_QCLAMP;"),
    ("hash_match_always", "if (same_coords(g->cells[e].c, c, g->d)) return e;", "return e;"),
    ("layers_count", "stats[0] = L + 1;", "stats[0] = L;"),
    ("median_upper_middle", "out = (float)(((double)v[size / 2 - 1] + (double)v[size / 2]) / 2.0);",
     "out = v[size / 2];"),
    ("median_natural_order",
     "uint32_t x = total_order_key(*(const float*)a), y = total_order_key(*(const float*)b);",
     "float x = *(const float*)a, y = *(const float*)b;"),
    ("median_sum_in_single", "out = (float)(((double)v[size / 2 - 1] + (double)v[size / 2]) / 2.0);",
     "out = (v[size / 2 - 1] + v[size / 2]) / 2.0f;"),
    ("buffer_keeps_k_plus", "if (*size == k && !entry_less(dist, id, buf[k - 1].dist, buf[k - 1].id)) return 0;",
     "if (*size == k && !entry_less(dist, id, buf[k - 1].dist, buf[k - 1].id)) return 1;"),
]


def _run_pins(lib_path):
    env = dict(os.environ, GHN_ORACLE_LIB=lib_path)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes(tmp_path):
    out = str(tmp_path / "control.so")
    compile_c(SRC, out)
    r = _run_pins(out)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,find,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, find, repl):
    with open(SRC) as f:
        src = f.read()
    assert src.count(find) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(find, repl))
    out = str(tmp_path / f"{name}.so")
    compile_c(str(path), out)
    r = _run_pins(out)
    assert r.returncode != 0, f"mutant {name} survived the pins"
