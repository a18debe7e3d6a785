"""Planted mistakes in a copy of the oracle, on the CPU: each plausible slip
(a dropped term, a flipped sign or comparison, an off-by-one) must make at least
one pin of tests/test_oracle_pins.py fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "dropped_pickup_to_dropoff_leg": ("oracle_leg(px, py, qx, qy) + ", ""),
    "exclusive_range": ("if (c <= R) { *cov = 1; *dist = c; }", "if (c < R) { *cov = 1; *dist = c; }"),
    "best_two_tie_high_index": ("(c == c1 && o < i1)", "(c == c1 && o > i1)"),
    "gain_sign": ("t->gd[j] += fxd - fad;", "t->gd[j] += fad - fxd;"),
    "extra_min_for_max": ("int32_t y = x > am ? x : am;", "int32_t y = x < am ? x : am;"),
    "loss_sign": ("t->ld[i] += fbd - fad;", "t->ld[i] += fad - fbd;"),
    "tenure_off_by_one": ("expiry[mi] = t + io->tenure + 1;", "expiry[mi] = t + io->tenure;"),
    "no_aspiration": ("int admissible = !tabu || better(c, d, best_c, best_d);", "int admissible = !tabu;"),
    "rank_tie_high_index": ("return a < b ? -1 : (a > b ? 1 : 0);", "return a > b ? -1 : (a < b ? 1 : 0);"),
    "move_tie_high_j": ("(c == ac && d == ad && (i < ai || (i == ai && j < aj)))",
                        "(c == ac && d == ad && (i < ai || (i == ai && j > aj)))"),
    "distance_before_coverage": ("if (c1 != c2) return c1 > c2;\n    return d1 < d2;",
                                 "if (d1 != d2) return d1 < d2;\n    return c1 > c2;"),
    "ceil_dropped": ("return (int32_t)ceil(d);", "return (int32_t)d;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", str(mutant),
                    "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
