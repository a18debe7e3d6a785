"""Planted mistakes in a copy of the oracle, on the CPU: each plausible slip
(a dropped term, a flipped sign or comparison, an off-by-one) must make at least
one pin fail -- of tests/test_oracle_pins.py for the C part (oracle.c), of
tests/test_oracle_haversine.py for its Haversine leg (Eq. 1), of
tests/test_oracle_fleet.py and tests/test_oracle_resume.py for the Python parts
(the heterogeneous fleet, the forced moves of reading A15), of
tests/test_oracle_local.py for the local search (Alg. 2)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")

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


# the Haversine leg of Eq. 1 and the table built from it
GEO_MUTANTS = {
    "haversine_no_latitude_factor": ("(cos(phi1) * cos(phi2)) * (sl * sl)", "(sl * sl)"),
    "haversine_full_angles": ("double sp = sin(0.5 * dphi), sl = sin(0.5 * dpsi);",
                              "double sp = sin(dphi), sl = sin(dpsi);"),
    "haversine_radius_not_doubled": ("(2.0 * ORACLE_EARTH_RADIUS_M) * asin", "ORACLE_EARTH_RADIUS_M * asin"),
    "haversine_longitude_from_latitudes": ("double dpsi = (double)(lon2 - lon1)",
                                           "double dpsi = (double)(lat2 - lat1)"),
    "haversine_rounded_down": ("asin(sqrt(h));\n    return (int32_t)ceil(d);",
                               "asin(sqrt(h));\n    return (int32_t)floor(d);"),
    "geo_dropped_return_leg": (" +\n               oracle_leg_haversine(qx, qy, bx, by)", ""),
}


def _c_mutant_survives(name, old, new, pin_files, tmp_path, exact_once=False):
    src = open(SRC).read()
    if exact_once:
        assert src.count(old) == 1, f"mutation site of {name} not found once"
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", str(mutant),
                    "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(ROOT, "tests", f) for f in pin_files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    survived, out = _c_mutant_survives(name, old, new, ("test_oracle_pins.py",), tmp_path)
    assert not survived, f"mutant {name} survived the pins:\n{out}"


@pytest.mark.parametrize("name", sorted(GEO_MUTANTS))
def test_haversine_pins_catch_mutant(name, tmp_path):
    old, new = GEO_MUTANTS[name]
    survived, out = _c_mutant_survives(name, old, new, ("test_oracle_haversine.py",), tmp_path, exact_once=True)
    assert not survived, f"mutant {name} survived the pins:\n{out}"


# the fleet ranking (Alg. 1, lines 14-16 and 20-21) and the fleet move rule (Sec. 3)
PY_MUTANTS = {
    "fleet_rank_reversed_order": ("key=lambda b: (int(S[b]), b))", "key=lambda b: (-int(S[b]), b))"),
    "fleet_rank_tie_high_index": ("key=lambda b: (int(S[b]), b))", "key=lambda b: (int(S[b]), -b))"),
    "fleet_rank_no_helipad_quota": ("            if nh < K_rotary:\n", "            if True:\n"),
    "fleet_rotary_takes_worst_aerodromes": (
        "rot += aer[:K_rotary - len(rot)]\n    fix = aer[K_rotary - nh:]",
        "rot += aer[len(aer) - (K_rotary - nh):]\n    fix = aer[:len(aer) - (K_rotary - nh)]"),
    "fleet_rotary_moves_first_on_ties": ("keys.append(((-f[0], f[1], i, j),", "keys.append(((-f[0], f[1], kind, i, j),"),
    "fleet_fixed_wing_on_helipad": ("if kind == 1 and heli[j]:", "if kind == 1 and heli[j] and False:"),
    "fleet_rotary_only_missions_by_any": ("b = evaluate(c1, r, R) if (c1.shape[1] and r)",
                                          "b = evaluate(c1, r + f, R) if (c1.shape[1] and r)"),
    "fleet_tenure_off_by_one": ("expiry[i] = expiry[j] = t + tenure + 1", "expiry[i] = expiry[j] = t + tenure"),
    "fleet_no_aspiration": ("adm = [k for k in keys if not k[6] or better(k[1], best)]",
                            "adm = [k for k in keys if not k[6]]"),
    # forced moves (reading A15)
    "forced_move_tie_high_j": ("key = (-cov, dist, j)", "key = (-cov, dist, -j)"),
    "forced_move_expiry_off_by_one": ("exp[i] = exp[j] = t + tenure", "exp[i] = exp[j] = t + tenure + 1"),
    "forced_moves_descending_ids": ("        i = out[0]\n", "        i = out[-1]\n"),
}
PY_PIN_FILES = ("test_oracle_fleet.py", "test_oracle_resume.py")

# the local search (Alg. 2 as read for identical vehicles): scan order,
# candidate bookkeeping, the table of the current placement, strictness, the
# local-optimum report
LS_MUTANTS = {
    "ls_closed_base_not_repositioned": ("O[s], cand[c] = j, i", "O[s] = j"),
    "ls_scan_slots_inside": ("s, c = int(pa[u // nC]), int(pb[u % nC])", "s, c = int(pa[u % K]), int(pb[u // K])"),
    "ls_table_kept_after_a_move": ("                moved = True\n                table = None\n",
                                   "                moved = True\n"),
    "ls_accepts_equal_objective": ("            if better(F, cur):\n", "            if not better(cur, F):\n"),
    "ls_optimum_never_reported": ("        if not moved:\n            optimum = True\n",
                                  "        if not moved:\n            optimum = False\n"),
}


def _py_mutant_survives(name, old, new, pin_files, tmp_path, orc):
    src = open(PY_SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not found once"
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    (pkg / "__init__.py").write_text(src.replace(old, new))
    env = dict(os.environ, ORACLE_PY_OVERRIDE=str(tmp_path), ORACLE_LIB_OVERRIDE=orc.build())
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(ROOT, "tests", f) for f in pin_files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_fleet_pins_catch_mutant(name, tmp_path, orc):
    old, new = PY_MUTANTS[name]
    survived, out = _py_mutant_survives(name, old, new, PY_PIN_FILES, tmp_path, orc)
    assert not survived, f"mutant {name} survived the pins:\n{out}"


@pytest.mark.parametrize("name", sorted(LS_MUTANTS))
def test_local_search_pins_catch_mutant(name, tmp_path, orc):
    old, new = LS_MUTANTS[name]
    survived, out = _py_mutant_survives(name, old, new, ("test_oracle_local.py",), tmp_path, orc)
    assert not survived, f"mutant {name} survived the pins:\n{out}"


def test_fleet_mutant_harness_runs_the_copy(tmp_path, orc):
    """The unmutated copy passes (so a failing mutant fails for its mutation)."""
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    (pkg / "__init__.py").write_text(open(PY_SRC).read() + "\nCOPY_MARK = 1\n")
    env = dict(os.environ, ORACLE_PY_OVERRIDE=str(tmp_path), ORACLE_LIB_OVERRIDE=orc.build())
    r = subprocess.run([sys.executable, "-c", "import sys; sys.path.insert(0, 'tests'); import conftest, oracle; "
                        "print(oracle.COPY_MARK)"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.stdout.strip() == "1", r.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(ROOT, "tests", f) for f in PY_PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
