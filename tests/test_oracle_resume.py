"""Pins of the oracle's forced moves (reading A15: an open base an update made
unavailable is closed, opening the available closed base with the best swap
objective) and of resuming a search from a kept state.

* hand-worked choices (the objectives worked out in the comments);
* numpy brute force: a forced move's placement beats (or ties with a higher
  id) every other available replacement, evaluated from scratch;
* order and bookkeeping: unavailable bases taken in ascending id, both bases
  of each move get expiry t + tenure, nothing else changes;
* resuming with no update equals the uninterrupted search.
"""
import numpy as np
import pytest

from test_oracle_pins import random_instance, table


def F_numpy(cost, open_, R):
    best = cost[np.asarray(open_)].min(axis=0).astype(np.int64)
    ok = best <= R
    return int(ok.sum()), int(best[ok].sum())


def test_hand_worked_forced_moves(orc):
    # bases x missions; R = 50
    c = np.array([[20, 30, 40], [25, 35, 20], [30, 15, 45], [40, 25, 15], [15, 45, 60]], np.int32)
    avail = np.array([1, 1, 1, 0, 1], np.uint8)
    # open {1, 3}, base 3 unavailable; candidates 0, 2, 4:
    #   {1, 0}: m0 min(25, 20) = 20, m1 min(35, 30) = 30, m2 min(20, 40) = 20 -> (3, 70)
    #   {1, 2}: m0 min(25, 30) = 25, m1 min(35, 15) = 15, m2 min(20, 45) = 20 -> (3, 60)
    #   {1, 4}: m0 min(25, 15) = 15, m1 min(35, 45) = 35, m2 min(20, 60) = 20 -> (3, 70)
    # -> open 2, at (3, 60)
    O, exp, done = orc.forced_moves(c, [1, 3], 50, avail, 7, 3, np.zeros(5, int))
    assert O == [1, 2] and done == [(3, 2, 3, 60)]
    assert exp.tolist() == [0, 0, 10, 10, 0]
    # ties: {1, 0} and {1, 4} both give (3, 70) once base 2 is gone too -> the lower id, 0
    avail2 = np.array([1, 1, 0, 0, 1], np.uint8)
    O, _, done = orc.forced_moves(c, [1, 3], 50, avail2, 0, 1, np.zeros(5, int))
    assert O == [1, 0] and done == [(3, 0, 3, 70)]
    # two unavailable open bases {2, 3}, ascending id: base 2 first.
    #   close 2 (open {3} kept): {0, 3}: m0 20, m1 25, m2 15 -> (3, 60); {1, 3}: 25, 25, 15 -> (3, 65);
    #   {4, 3}: 15, 25, 15 -> (3, 55)  -> open 4
    #   close 3 (open {4} kept): {4, 0}: 15, 30, 40 -> (3, 85); {4, 1}: 15, 35, 20 -> (3, 70) -> open 1
    avail3 = np.array([1, 1, 0, 0, 1], np.uint8)
    O, exp, done = orc.forced_moves(c, [2, 3], 50, avail3, 4, 2, np.zeros(5, int))
    assert done == [(2, 4, 3, 55), (3, 1, 3, 70)] and O == [4, 1]
    assert exp.tolist() == [0, 6, 6, 6, 6]


@pytest.mark.parametrize("seed", range(8))
def test_forced_moves_against_bruteforce(orc, seed):
    inst = random_instance(700 + seed, B=14, M=50, K=4)
    cost = table(orc, inst)
    rng = np.random.default_rng(seed)
    open_ = [int(x) for x in rng.choice(inst.B, inst.K, replace=False)]
    avail = np.ones(inst.B, np.uint8)
    gone = rng.choice(open_, size=1 + seed % 2, replace=False)
    avail[gone] = 0
    expiry = rng.integers(0, 5, size=inst.B)
    O, exp, done = orc.forced_moves(cost, open_, inst.R, avail, 9, 3, expiry)
    assert [i for (i, _, _, _) in done] == sorted(int(g) for g in gone)
    cur = list(open_)
    for (i, j, cov, dist) in done:
        k = cur.index(i)
        options = []
        for b in range(inst.B):
            if avail[b] and b not in cur:
                trial = cur[:k] + [b] + cur[k + 1:]
                options.append(((-F_numpy(cost, trial, inst.R)[0], F_numpy(cost, trial, inst.R)[1], b), b))
        assert min(options)[1] == j
        cur[k] = j
        assert F_numpy(cost, cur, inst.R) == (cov, dist)
    assert cur == O and all(avail[b] for b in O) and len(set(O)) == inst.K
    moved = {x for (i, j, _, _) in done for x in (i, j)}
    for b in range(inst.B):
        assert exp[b] == (12 if b in moved else expiry[b])


@pytest.mark.parametrize("seed", range(4))
def test_resume_without_update_equals_uninterrupted(orc, seed):
    inst = random_instance(800 + seed, B=16, M=80, K=4)
    cost = table(orc, inst)
    full = orc.tabu(cost, inst.K, inst.R, 30, 3)
    first = orc.tabu(cost, inst.K, inst.R, 12, 3)
    # the kept state: final placement in slot order is not returned sorted by
    # the oracle, but the search does not depend on slot order
    rest = orc.tabu(cost, inst.K, inst.R, 18, 3, start_open=first.final_open, t0=12, expiry_in=first.expiry,
                    best_in=first.best_open, best_cov_in=first.best_cov, best_dist_in=first.best_dist,
                    best_iter_in=first.best_iter)
    assert first.moves + rest.moves == full.moves
    assert (rest.best_cov, rest.best_dist, rest.best_iter) == (full.best_cov, full.best_dist, full.best_iter)
