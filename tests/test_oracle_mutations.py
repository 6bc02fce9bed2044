"""Plant plausible mistakes in copies of the oracle (on the CPU) and require
the pins to catch every one: a dropped term, a wrong sign, an off-by-one, a
transposed operand, a reversed tie rule. This shows the pins constrain each
part of the oracle, not just its overall shape."""
import os
import subprocess
import sys

import pytest

import oracle
import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gumap_oracle.c")

# (name, original text, mutated text): each original must occur exactly once.
# The clamp max(0, d - rho) has no mutant here: rho is the row minimum, so the
# clamp never changes a value (an equivalent mutant, not a mistake).
MUTATIONS = [
    ("tie_rule_reversed", "return (x->v > y->v) - (x->v < y->v);", "return (x->v < y->v) - (x->v > y->v);"),
    ("bfs_step_two", "dist[w] = dist[u] + 1;", "dist[w] = dist[u] + 2;"),
    ("self_in_list", "if (v != s && dist[v] >= 0)", "if (dist[v] >= 0)"),
    ("partial_stops_early", "while (n_found < k && n_cur > 0)", "while (n_found < k - 1 && n_cur > 0)"),
    ("partial_level_offset", "found[n_found].d = level;", "found[n_found].d = level + 1;"),
    ("partial_work_skips_degree", "work += row_ptr[u + 1] - row_ptr[u];", "work += 1;"),
    ("weight_sign", "a[j] = isinf(sigma) ? 1.0 : exp(-x / sigma);", "a[j] = isinf(sigma) ? 1.0 : exp(x / sigma);"),
    ("rho_zero", "double rho = (double)d[0];", "double rho = 0.0;"),
    ("target_natural_log", "const double T = log2((double)k);", "const double T = log((double)k);"),
    ("floor_dropped", "if (sigma < floor_) sigma = floor_;", ""),
    ("floor_scale", "double floor_ = 1e-3 * mean;", "double floor_ = 1e-2 * mean;"),
    ("bisection_direction", "if (f_sigma(d, kv, rho, mid) > T) hi = mid;", "if (f_sigma(d, kv, rho, mid) < T) hi = mid;"),
    ("union_drops_product_coo", "v = v + e[q].val - v * e[q].val;", "v = v + e[q].val;"),
    ("union_drops_product_slot", "aij + aji - aij * aji", "aij + aji"),
    ("union_lookup_transposed", "lookup(idx, a, k, j, i)", "lookup(idx, a, k, i, j)"),
    ("coo_no_transpose", "e[m].key = (int64_t)j * n + i; e[m].val = v; m++;",
     "e[m].key = (int64_t)i * n + j; e[m].val = v; m++;"),
    ("no_root_small_row", "if ((double)kv <= T) {", "if ((double)kv < 0.0) {"),
    ("np_self_in_ball", "if (u != v && dist[u] >= 0 && dist[u] <= r) c++;", "if (dist[u] >= 0 && dist[u] <= r) c++;"),
    ("np_radius_short", "if (u != v && dist[u] >= 0 && dist[u] <= r) c++;",
     "if (u != v && dist[u] >= 0 && dist[u] < r) c++;"),
    ("np_geo_tie_reversed", "return x->v < y->v ? -1 : (x->v > y->v);", "return x->v > y->v ? -1 : (x->v < y->v);"),
    ("np_union_size", "(double)inter / (double)(2 * c - inter)", "(double)inter / (double)(2 * c)"),
    ("np_unsquared", "float sq = dx * dx;", "float sq = dx;"),
    ("np_empty_ball_zero", "total += c == 0 ? 1.0 :", "total += c == 0 ? 0.0 :"),
    ("stress_normalisation", "return total / ((double)n * (double)n - (double)n);", "return total / ((double)n * (double)n);"),
    ("stress_unreachable_zero", "if (dist[j] < 0) { row += 1.0; continue; }", "if (dist[j] < 0) { continue; }"),
    ("stress_no_sqrt", "double t = ((double)dist[j] - sqrt(sq)) / (double)dist[j];",
     "double t = ((double)dist[j] - sq) / (double)dist[j];"),
    ("stress_not_relative", "double t = ((double)dist[j] - sqrt(sq)) / (double)dist[j];",
     "double t = ((double)dist[j] - sqrt(sq));"),
]


RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, oracle_pins as pins
orc = oracle.Oracle({lib!r})
for check in pins.ALL_CHECKS:
    try:
        check(orc)
    except Exception as e:
        print("caught by", check.__name__, type(e).__name__)
        sys.exit(3)
print("not caught")
"""


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(tmp_path, name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / f"oracle_{name}.c"
    mutated.write_text(text.replace(old, new))
    lib = oracle.compile_source(str(mutated), str(tmp_path / f"lib_{name}.so"))
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    code = RUNNER.format(root=os.path.dirname(tests_dir), tests=tests_dir, lib=lib)
    try:
        proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=20)
    except subprocess.TimeoutExpired:
        return  # the planted mistake makes the oracle hang: caught
    assert proc.returncode != 0, f"planted mistake '{name}' passed every pin: {proc.stdout}"


# Planted mistakes in the spectral-layout oracle (oracle/spectral.py). The
# sign convention of each column has no mutant: the pins compare up to sign,
# as the definition fixes eigenvectors only up to sign.
SPECTRAL_SRC = os.path.join(os.path.dirname(oracle.__file__), "spectral.py")
SPECTRAL_MUTATIONS = [
    ("combinatorial_laplacian", "L_sym = np.eye(m) - (s[:, None] * Wl) * s[None, :]", "L_sym = np.diag(deg[live]) - Wl"),
    ("no_degree_scaling", "Xl = Y * s[:, None]", "Xl = Y.copy()"),
    ("skips_one_more", "Y = evecs[:, :take]", "Y = evecs[:, 1:take + 1]"),
    ("trivial_kept", "Z = Z - np.outer(t, t @ Z)", "Z = Z + 0.0"),
    ("unit_degrees", "deg = W.sum(axis=1)", "deg = (W > 0).sum(axis=1).astype(np.float64)"),
    ("largest_instead", "evals, evecs = np.linalg.eigh(L_sym)", "evals, evecs = np.linalg.eigh(-L_sym); evals = -evals"),
]

SPECTRAL_RUNNER = """
import importlib.util, sys
sys.path[:0] = [{root!r}, {tests!r}]
import spectral_pins as spins
spec = importlib.util.spec_from_file_location("spectral_mutant", {path!r})
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
for check in spins.ALL_CHECKS:
    try:
        check(mod)
    except Exception as e:
        print("caught by", check.__name__, type(e).__name__)
        sys.exit(3)
print("not caught")
"""


@pytest.mark.parametrize("name,old,new", SPECTRAL_MUTATIONS, ids=[m[0] for m in SPECTRAL_MUTATIONS])
def test_spectral_mutation_is_caught(tmp_path, name, old, new):
    with open(SPECTRAL_SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / f"spectral_{name}.py"
    mutated.write_text(text.replace(old, new))
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    code = SPECTRAL_RUNNER.format(root=os.path.dirname(tests_dir), tests=tests_dir, path=str(mutated))
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=60)
    assert proc.returncode != 0, f"planted mistake '{name}' passed every pin: {proc.stdout}"
