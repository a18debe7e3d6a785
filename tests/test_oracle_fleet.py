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
  rule; the best found is never better than the exhaustive optimum;
* a hand-worked instance (tests/golden/fleet_hand_worked.json): the ranking
  with the helipad rule for several fleet mixes, and a 3-move trajectory;
* an independent brute-force replay, written from the paper and sharing
  nothing with the oracle, on 36 tiny fleets with many ties: the ranking
  (Alg. 1 with the helipad quota of lines 14-16 and the vehicle assignment of
  lines 20-21) and the search (every vehicle's moves to every compatible closed
  base evaluated from scratch, mission by mission; tabu, aspiration, fallback,
  the (covered desc, distance asc, vacated base asc, opened base asc) order).
"""
import itertools
import json
import os

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


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fleet_hand_worked.json")


@pytest.fixture(scope="module")
def fleet_golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_golden_fleet_rank(orc, fleet_golden):
    g = fleet_golden
    c = np.array(g["cost"], dtype=np.int32)
    heli = np.array(g["helipad"], bool)
    assert c.astype(np.int64).sum(axis=1).tolist() == g["rowsum"]
    for case in g["rank"]["cases"]:
        av = None if "avail" not in case else np.array(case["avail"], np.uint8)
        rot, fix = orc.fleet_rank(c, heli, case["K_rotary"], case["K_fixed"], av)
        assert (list(rot), list(fix)) == (case["rotary"], case["fixed"]), case


def test_golden_fleet_tabu(orc, fleet_golden):
    g = fleet_golden
    c = np.array(g["cost"], dtype=np.int32)
    heli = np.array(g["helipad"], bool)
    rmask = np.array(g["mission_rotary"], bool)
    t = g["tabu"]
    zero = orc.fleet_tabu(c, heli, rmask, t["K_rotary"], t["K_fixed"], t["R"], 0, t["tenure"])
    assert (zero.final_cov, zero.final_dist) == (t["start"]["cov"], t["start"]["dist"])
    assert zero.final_rotary.tolist() == t["start"]["rotary"] and zero.final_fixed.tolist() == t["start"]["fixed"]
    for mode in ("full", "table"):
        r = orc.fleet_tabu(c, heli, rmask, t["K_rotary"], t["K_fixed"], t["R"], t["iters"], t["tenure"],
                           eval_mode=mode)
        assert [list(m) for m in r.moves] == t["moves"], mode
        assert r.best_rotary.tolist() == t["best_rotary"] and r.best_fixed.tolist() == t["best_fixed"]
        assert (r.best_cov, r.best_dist, r.best_iter) == (t["best_cov"], t["best_dist"], t["best_iter"])
        assert r.final_rotary.tolist() == t["final_rotary"] and r.final_fixed.tolist() == t["final_fixed"]
        imp = orc.fleet_tabu(c, heli, rmask, t["K_rotary"], t["K_fixed"], t["R"], t["iters"], t["tenure"],
                             accept_worsening=False, eval_mode=mode)
        assert [list(m) for m in imp.moves] == t["improving_only_moves"], mode


# ---- independent replay (plain Python, mission by mission) ----

def replay_objective(cost, rmask, rot, fix, R):
    """Eq. 2 with Eq. 10: each mission from its nearest open base that may fly
    it (a rotary-only mission from a base holding a rotary-wing vehicle)."""
    cov = dist = 0
    for m in range(len(rmask)):
        best = None
        for b in (rot if rmask[m] else rot + fix):
            c = int(cost[b][m])
            if best is None or c < best:
                best = c
        if best is not None and best <= R:
            cov += 1
            dist += best
    return cov, dist


def replay_rank(cost, heli, K_rotary, K_fixed, avail):
    """Alg. 1 with the helipad quota, restated: the chosen bases are the best
    K_rotary + K_fixed, by (row sum over all missions, id), among the available
    aerodromes and the K_rotary best available helipads.  Helipads take
    rotary-wing vehicles; the best-ranked chosen aerodromes take the remaining
    rotary-wing vehicles, the others the fixed-wing ones."""
    B = len(heli)
    S = [sum(int(x) for x in cost[b]) for b in range(B)]

    def take_best(pool):
        b = pool[0]
        for x in pool[1:]:
            if S[x] < S[b] or (S[x] == S[b] and x < b):
                b = x
        pool.remove(b)
        return b

    helis = [b for b in range(B) if avail[b] and heli[b]]
    cand = [b for b in range(B) if avail[b] and not heli[b]]
    for _ in range(min(K_rotary, len(helis))):
        cand.append(take_best(helis))
    chosen = [take_best(cand) for _ in range(min(K_rotary + K_fixed, len(cand)))]
    rot = [b for b in chosen if heli[b]]
    aer = [b for b in chosen if not heli[b]]
    need = K_rotary - len(rot)
    if need < 0 or len(aer) - need != K_fixed:
        raise ValueError("infeasible")
    return rot + aer[:need], aer[need:]


def replay_tabu(cost, heli, rmask, rot, fix, R, iters, tenure, avail, accept_worsening=True):
    B = len(heli)
    rot, fix = list(rot), list(fix)
    cur = replay_objective(cost, rmask, rot, fix, R)
    best = cur
    expiry = [0] * B
    moves = []

    def better(x, y):
        return x[0] > y[0] or (x[0] == y[0] and x[1] < y[1])

    for t in range(iters):
        top_all = top_adm = None
        for kind, group in ((0, rot), (1, fix)):
            for sl, i in enumerate(group):
                for j in range(B):
                    if not avail[j] or j in rot or j in fix or (kind == 1 and heli[j]):
                        continue
                    r2, f2 = list(rot), list(fix)
                    (r2 if kind == 0 else f2)[sl] = j
                    v = replay_objective(cost, rmask, r2, f2, R)
                    key = (-v[0], v[1], i, j)
                    tabu = t < expiry[i] or t < expiry[j]
                    item = (key, v, kind, sl, tabu)
                    if top_all is None or key < top_all[0]:
                        top_all = item
                    if (not tabu or better(v, best)) and (top_adm is None or key < top_adm[0]):
                        top_adm = item
        if top_all is None:
            break
        pick = top_adm if top_adm is not None else top_all
        flags = (2 if pick[4] else 0) if top_adm is not None else 1
        if not accept_worsening and not better(pick[1], cur):
            break
        (_, _, i, j), v, kind, sl, _ = pick
        (rot if kind == 0 else fix)[sl] = j
        expiry[i] = expiry[j] = t + tenure + 1
        cur = v
        if better(v, best):
            best = v
            flags |= 4
        moves.append((t, i, j, flags, v[0], v[1]))
    return moves, best


def tiny_fleet(seed):
    rng = np.random.default_rng(9000 + seed)
    B = int(rng.integers(5, 10))
    M = int(rng.integers(3, 11))
    cost = rng.integers(1, 13, size=(B, M)).astype(np.int32)   # small range: many ties
    heli = rng.random(B) < 0.4
    rmask = rng.random(M) < 0.3
    avail = np.ones(B, np.uint8)
    if seed % 3 == 0:
        avail[int(rng.integers(0, B))] = 0
    K_rotary = int(rng.integers(0, 4))
    K_fixed = int(rng.integers(0, 4))
    if K_rotary + K_fixed == 0:
        K_fixed = 1
    while K_rotary + K_fixed > B - 2:
        if K_fixed:
            K_fixed -= 1
        else:
            K_rotary -= 1
    R = int(rng.integers(4, 13))
    tenure = int(rng.integers(0, 4))
    return cost, heli, rmask, avail, K_rotary, K_fixed, R, tenure


@pytest.mark.parametrize("seed", range(36))
def test_fleet_matches_bruteforce_replay(orc, seed):
    cost, heli, rmask, avail, Kr, Kf, R, tenure = tiny_fleet(seed)
    try:
        want_rot, want_fix = replay_rank(cost, heli, Kr, Kf, avail)
    except ValueError:
        with pytest.raises(ValueError):
            orc.fleet_rank(cost, heli, Kr, Kf, avail)
        return
    rot, fix = orc.fleet_rank(cost, heli, Kr, Kf, avail)
    assert sorted(rot) == sorted(want_rot) and sorted(fix) == sorted(want_fix)
    # from the ranking, and from a random compatible start
    rng = np.random.default_rng(seed)
    perm = [int(b) for b in rng.permutation(len(heli)) if avail[b]]
    s_fix = [b for b in perm if not heli[b]][:Kf]
    s_rot = [b for b in perm if b not in s_fix][:Kr]
    starts = [(want_rot, want_fix)]
    if len(s_fix) == Kf and len(s_rot) == Kr:
        starts.append((s_rot, s_fix))
    for srot, sfix in starts:
        for worsen in (True, False):
            want, best = replay_tabu(cost, heli, rmask, srot, sfix, R, 12, tenure, avail, worsen)
            for mode in ("full", "table"):
                got = orc.fleet_tabu(cost, heli, rmask, Kr, Kf, R, 12, tenure, start_rotary=srot, start_fixed=sfix,
                                     avail=avail, accept_worsening=worsen, eval_mode=mode)
                assert [tuple(int(x) for x in m) for m in got.moves] == want, (mode, worsen)
                assert (got.best_cov, got.best_dist) == best


def test_replay_sees_ties_between_vehicle_kinds():
    """The tiny fleets exercise the tie order: in some step a rotary-wing and a
    fixed-wing move reach the same objective."""
    seen = 0
    for seed in range(36):
        cost, heli, rmask, avail, Kr, Kf, R, tenure = tiny_fleet(seed)
        try:
            rot, fix = replay_rank(cost, heli, Kr, Kf, avail)
        except ValueError:
            continue
        if not rot or not fix:
            continue
        vals = {}
        for kind, group in ((0, rot), (1, fix)):
            for sl, i in enumerate(group):
                for j in range(len(heli)):
                    if not avail[j] or j in rot or j in fix or (kind == 1 and heli[j]):
                        continue
                    r2, f2 = list(rot), list(fix)
                    (r2 if kind == 0 else f2)[sl] = j
                    vals.setdefault(replay_objective(cost, rmask, r2, f2, R), set()).add(kind)
        seen += any(len(k) == 2 for k in vals.values())
    assert seen >= 5
