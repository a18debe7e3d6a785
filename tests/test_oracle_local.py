"""Pins of the oracle's local search (Alg. 2 as read for identical vehicles).

* the table form (one fast-interchange table per placement) against the plain
  definition (every pair judged by evaluating the swapped placement afresh);
* an independent replay in Python: the scan order, the first-improvement rule
  and the candidate-position bookkeeping, with numpy objectives;
* invariants: every move strictly improves and its objective equals a
  recomputation; moves within a pass come in increasing scan order; a reported
  local optimum admits no improving swap at all (checked by brute force); a
  start that is already the exhaustive optimum makes no move.
"""
import numpy as np
import pytest

from paper_2001_05291_gb300 import synth

from test_oracle_pins import F_numpy, random_instance, table


def better(x, y):
    return x[0] > y[0] or (x[0] == y[0] and x[1] < y[1])


def replay_numpy(cost, K, R, ps, pc, start, avail=None, max_moves=10**9):
    """The same rules written out again over numpy objectives (no oracle call)."""
    B = cost.shape[0]
    O = [int(x) for x in start]
    av = np.ones(B, bool) if avail is None else np.asarray(avail, bool)
    cand = [b for b in range(B) if av[b] and b not in set(O)]
    nC = len(cand)
    cur = F_numpy(cost, O, R)
    moves, passes, optimum = [], 0, False
    if nC == 0:
        return moves, O, cur, 0, True
    for p in range(len(ps)):
        passes += 1
        moved = False
        for a in range(K):
            for b in range(nC):
                if len(moves) >= max_moves:
                    break
                s, c = int(ps[p][a]), int(pc[p][b])
                trial = list(O)
                trial[s] = cand[c]
                F = F_numpy(cost, trial, R)
                if better(F, cur):
                    moves.append((len(moves), O[s], cand[c], 4, F[0], F[1]))
                    O[s], cand[c] = cand[c], O[s]
                    cur, moved = F, True
        if len(moves) >= max_moves:
            break
        if not moved:
            optimum = True
            break
    return moves, O, cur, passes, optimum


@pytest.mark.parametrize("seed", range(12))
def test_table_form_equals_plain_definition_and_replay(orc, seed):
    inst = random_instance(700 + seed)
    cost = table(orc, inst)
    K, R = inst.K, inst.R
    nC = inst.B - K
    ps, pc = synth.scan_orders(seed, 4, K, nC)
    start, _ = orc.rank(cost, K)
    full = orc.local_search(cost, K, R, ps, pc, eval_mode="full")
    tab = orc.local_search(cost, K, R, ps, pc, eval_mode="table")
    assert full.moves == tab.moves and np.array_equal(full.final_open, tab.final_open)
    assert (full.final_cov, full.final_dist, full.passes, full.local_optimum) == \
        (tab.final_cov, tab.final_dist, tab.passes, tab.local_optimum)
    moves, O, cur, passes, optimum = replay_numpy(cost, K, R, ps, pc, start)
    assert tab.moves == moves
    assert np.array_equal(tab.final_open, np.sort(O))
    assert (tab.final_cov, tab.final_dist) == cur
    assert (tab.passes, tab.local_optimum) == (passes, optimum)


@pytest.mark.parametrize("seed", range(6))
def test_moves_improve_in_scan_order_and_optimum_is_local(orc, seed):
    inst = random_instance(900 + seed, B=14, M=60, K=4)
    cost = table(orc, inst)
    K, R = inst.K, inst.R
    nC = inst.B - K
    ps, pc = synth.scan_orders(100 + seed, 6, K, nC)
    res = orc.local_search(cost, K, R, ps, pc)
    start, _ = orc.rank(cost, K)
    O = [int(x) for x in start]
    cand = [b for b in range(inst.B) if b not in set(O)]
    prev = orc.evaluate(cost, O, R)
    # replay: every move strictly better, equal to a recomputation, at a scan
    # position after the previous move of the same pass
    pass_of_move = []
    p, last_u = 0, -1
    for (n, i, j, flags, cov, dist) in res.moves:
        s, c = O.index(i), cand.index(j)
        while True:
            rs = {int(v): a for a, v in enumerate(ps[p])}
            rc = {int(v): b for b, v in enumerate(pc[p])}
            u = rs[s] * nC + rc[c]
            if u > last_u:
                break
            p, last_u = p + 1, -1
        last_u = u
        pass_of_move.append(p)
        O[s], cand[c] = j, i
        assert better((cov, dist), prev) and orc.evaluate(cost, O, R) == (cov, dist)
        prev = (cov, dist)
    assert pass_of_move == sorted(pass_of_move)
    if res.local_optimum:
        for s in range(K):
            for j in cand:
                trial = list(O)
                trial[s] = j
                assert not better(orc.evaluate(cost, trial, R), prev)


def test_start_at_the_exhaustive_optimum_makes_no_move(orc):
    inst = random_instance(31, B=10, M=40, K=3)
    cost = table(orc, inst)
    opt, oc, od, _ = orc.bruteforce(cost, 3, inst.R)
    ps, pc = synth.scan_orders(5, 3, 3, inst.B - 3)
    res = orc.local_search(cost, 3, inst.R, ps, pc, start_open=opt)
    assert res.moves == [] and res.local_optimum and res.passes == 1
    assert (res.final_cov, res.final_dist) == (oc, od)


def test_budget_and_passes_run_out(orc):
    inst = random_instance(41, B=15, M=80, K=4)
    cost = table(orc, inst)
    nC = inst.B - 4
    ps, pc = synth.scan_orders(9, 5, 4, nC)
    full = orc.local_search(cost, 4, inst.R, ps, pc)
    assert len(full.moves) >= 2
    cut = orc.local_search(cost, 4, inst.R, ps, pc, max_moves=1)
    assert cut.moves == full.moves[:1] and not cut.local_optimum
    one = orc.local_search(cost, 4, inst.R, ps[:1], pc[:1])
    assert one.passes == 1 and one.moves == [m for m in full.moves][:len(one.moves)]


def test_unavailable_bases_never_open(orc):
    inst = random_instance(51, B=14, M=70, K=4)
    cost = table(orc, inst)
    avail = np.ones(inst.B, np.uint8)
    avail[[2, 7]] = 0
    start, _ = orc.rank(cost, 4, avail)
    nC = int(avail.sum()) - 4
    ps, pc = synth.scan_orders(11, 4, 4, nC)
    res = orc.local_search(cost, 4, inst.R, ps, pc, avail=avail)
    moves, O, cur, passes, optimum = replay_numpy(cost, 4, inst.R, ps, pc, start, avail)
    assert res.moves == moves and (res.passes, res.local_optimum) == (passes, optimum)
    assert all(j not in (2, 7) for (_, _, j, *_r) in res.moves)


def test_scan_orders_are_permutations():
    ps, pc = synth.scan_orders(3, 5, 7, 30)
    for p in range(5):
        assert sorted(ps[p]) == list(range(7)) and sorted(pc[p]) == list(range(30))
    assert not np.array_equal(ps[0], ps[1]) or not np.array_equal(pc[0], pc[1])
