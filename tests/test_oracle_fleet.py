"""Pins of the oracle's heterogeneous-fleet search (rotary- and fixed-wing
vehicles, helipads, rotary-only missions).

* reductions to the identical-vehicle search, which has its own pins: with no
  fixed-wing vehicle, and with no helipad and no rotary-only mission, the
  trajectory equals tabu()'s;
* the table form equals the plain form (every move's placement evaluated from
  scratch);
* the objective written out in numpy (each mission's nearest compatible open
  base) equals every recorded objective along the replayed trajectory;
* fixed-wing vehicles never stand at a helipad; the ranking obeys the helipad
  rule; the best found is never better than the exhaustive optimum.
"""
import itertools

import numpy as np
import pytest

from test_oracle_pins import random_instance, table


def fleet_F_numpy(cost, rmask, rot, fix, R):
    """Covered count and distance with each mission at its nearest compatible open base."""
    allb = cost[np.asarray(list(rot) + list(fix))].min(axis=0)
    if rot:
        rb = cost[np.asarray(list(rot))].min(axis=0)
        best = np.where(rmask, rb, allb)
        cov_ok = np.ones_like(rmask)
    else:
        best = allb
        cov_ok = ~rmask            # rotary-only missions cannot be flown
    ok = (best <= R) & cov_ok
    return int(ok.sum()), int(best[ok].astype(np.int64).sum())


def setup(orc, seed, B=14, M=60, heli_ids=(1, 4, 9), rot_every=5):
    inst = random_instance(seed, B=B, M=M, K=4)
    cost = table(orc, inst)
    heli = np.zeros(inst.B, bool)
    heli[list(heli_ids)] = True
    rmask = np.zeros(inst.M, bool)
    rmask[::rot_every] = True
    return inst, cost, heli, rmask


@pytest.mark.parametrize("seed", range(4))
def test_reduces_to_identical_vehicles(orc, seed):
    inst, cost, heli, rmask = setup(orc, 300 + seed)
    plain = orc.tabu(cost, 4, inst.R, 25, 3)
    allrot = orc.fleet_tabu(cost, heli, rmask, 4, 0, inst.R, 25, 3)
    assert allrot.moves == plain.moves
    none = np.zeros(inst.B, bool)
    mixed = orc.fleet_tabu(cost, none, np.zeros(inst.M, bool), 2, 2, inst.R, 25, 3)
    assert mixed.moves == plain.moves


@pytest.mark.parametrize("seed", range(6))
def test_table_form_objective_and_rules(orc, seed):
    inst, cost, heli, rmask = setup(orc, 400 + seed)
    full = orc.fleet_tabu(cost, heli, rmask, 2, 2, inst.R, 30, 3)
    tab = orc.fleet_tabu(cost, heli, rmask, 2, 2, inst.R, 30, 3, eval_mode="table")
    assert full.moves == tab.moves
    rot, fix = orc.fleet_rank(cost, heli, 2, 2)
    assert sum(heli[b] for b in rot + fix) <= 2 and not any(heli[b] for b in fix)
    start = fleet_F_numpy(cost, rmask, rot, fix, inst.R)
    zero = orc.fleet_tabu(cost, heli, rmask, 2, 2, inst.R, 0, 3)
    assert (zero.final_cov, zero.final_dist) == start
    rot, fix = list(rot), list(fix)
    for (t, i, j, flags, cov, dist) in full.moves:
        if i in rot:
            rot[rot.index(i)] = j
        else:
            assert not heli[j]
            fix[fix.index(i)] = j
        assert fleet_F_numpy(cost, rmask, rot, fix, inst.R) == (cov, dist)
    assert not any(heli[b] for b in fix)
    assert (full.best_cov, -full.best_dist) >= (start[0], -start[1])


def test_best_not_above_exhaustive_optimum(orc):
    inst, cost, heli, rmask = setup(orc, 500, B=9, M=40, heli_ids=(2, 6), rot_every=4)
    res = orc.fleet_tabu(cost, heli, rmask, 2, 1, inst.R, 40, 2)
    best = None
    for rot in itertools.combinations(range(inst.B), 2):
        for f in range(inst.B):
            if f in rot or heli[f]:
                continue
            v = fleet_F_numpy(cost, rmask, list(rot), [f], inst.R)
            if best is None or (v[0], -v[1]) > (best[0], -best[1]):
                best = v
    assert (res.best_cov, -res.best_dist) <= (best[0], -best[1])


def test_no_rotary_vehicle_leaves_rotary_only_missions_uncovered(orc):
    inst, cost, heli, rmask = setup(orc, 600)
    res = orc.fleet_tabu(cost, heli, rmask, 0, 3, inst.R, 10, 2)
    assert res.best_cov <= int((~rmask).sum())
    assert not any(heli[b] for b in res.final_fixed)
