"""Pins of the incremental form of the swap neighbourhood, on the CPU and
without the GPU code.

For tables beyond L2 the GPU keeps the fast-interchange terms (gain[j],
extra[i][j]) across Tabu moves instead of recomputing them: a move changes them
only through the missions whose clamped best / second-best cost or (while
covered) best slot changed -- their old terms come out of every column and
their new terms go in -- and through the closed base, a candidate again, whose
column is rebuilt over every mission.  Along oracle Tabu trajectories this file
applies exactly that rule in numpy and checks, after every move:

* the kept terms equal the terms recomputed from scratch for the new placement
  on every candidate column;
* V0 + gain[j] + loss[i] + extra[i][j] equals the oracle's direct evaluation of
  every swap (i, j) (a different computation: the placement after the swap,
  evaluated mission by mission);
* leaving out either half of the rule (the closed column's rebuild, or taking
  the old terms out) is caught.
"""
import numpy as np
import pytest

from test_oracle_pins import random_instance, table


def state(orc, cost, O, R):
    """Clamped best and second-best cost and best slot of every mission."""
    a, b, b1, _ = orc.best_two(cost, np.asarray(O, dtype=np.int32))
    pos = {int(base): k for k, base in enumerate(O)}
    s1 = np.array([pos[int(x)] for x in b1], dtype=np.int64)
    return np.minimum(a.astype(np.int64), R + 1), np.minimum(b.astype(np.int64), R + 1), s1


def terms(cost, a1, b1, s1, R, K):
    """gain (count, distance) per base and extra (count, distance) per (slot,
    base), summed over the given missions (columns of `cost`)."""
    x = cost.astype(np.int64)
    ca, cb = (a1 <= R).astype(np.int64), (b1 <= R).astype(np.int64)
    gh = x < a1
    gain_c = np.where(gh, 1 - ca, 0).sum(axis=1)
    gain_d = np.where(gh, x - np.where(ca == 1, a1, 0), 0).sum(axis=1)
    eh = x < b1
    ec = np.where(eh, ca - cb, 0)
    ed = np.where(eh, np.where(ca == 1, np.maximum(x, a1), 0) - np.where(cb == 1, b1, 0), 0)
    B = cost.shape[0]
    extra_c = np.zeros((K, B), dtype=np.int64)
    extra_d = np.zeros((K, B), dtype=np.int64)
    for k in range(K):
        sel = s1 == k
        extra_c[k] = ec[:, sel].sum(axis=1)
        extra_d[k] = ed[:, sel].sum(axis=1)
    return gain_c, gain_d, extra_c, extra_d


def loss_v0(a1, b1, s1, R, K):
    fa_c, fa_d = (a1 <= R).astype(np.int64), np.where(a1 <= R, a1, 0)
    fb_c, fb_d = (b1 <= R).astype(np.int64), np.where(b1 <= R, b1, 0)
    lc = np.array([(fb_c - fa_c)[s1 == k].sum() for k in range(K)])
    ld = np.array([(fb_d - fa_d)[s1 == k].sum() for k in range(K)])
    return int(fa_c.sum()), int(fa_d.sum()), lc, ld


def replay(orc, cost, K, R, moves, start, rebuild_closed=True, take_out_old=True):
    """Keep the terms along the moves by the incremental rule, as the GPU does:
    the first full pass fills the candidates' columns only, a move's update
    skips the closed base's column, which is zeroed and rebuilt over every
    mission.  After each move yield (placement, kept terms, new state)."""
    O = [int(x) for x in start]
    st = state(orc, cost, O, R)
    kept = list(terms(cost, *st, R, K))
    for q in range(2):
        kept[q][O] = 0
    for q in (2, 3):
        kept[q][:, O] = 0
    for (_, i, j, *_r) in moves:
        s = O.index(i)
        O[s] = j
        new = state(orc, cost, O, R)
        a0, b0, s0 = st
        a1, b1, s1 = new
        ch = (a0 != a1) | (b0 != b1) | ((a1 <= R) & (s0 != s1))
        add = terms(cost[:, ch], a1[ch], b1[ch], s1[ch], R, K)
        out = terms(cost[:, ch], a0[ch], b0[ch], s0[ch], R, K)
        keep_i = [kept[0][i], kept[1][i], kept[2][:, i].copy(), kept[3][:, i].copy()]
        for q in range(4):
            kept[q] = kept[q] + add[q] - (out[q] if take_out_old else 0)
        kept[0][i], kept[1][i], kept[2][:, i], kept[3][:, i] = keep_i   # not updated: rebuilt below
        if rebuild_closed:
            full = terms(cost[i:i + 1], a1, b1, s1, R, K)
            kept[0][i], kept[1][i] = full[0][0], full[1][0]
            kept[2][:, i], kept[3][:, i] = full[2][:, 0], full[3][:, 0]
        st = new
        yield list(O), kept, new


CASES = [(7001, 30, 900, 5, None), (7002, 45, 600, 8, 250_000), (7003, 25, 700, 1, None),
         (7004, 40, 800, 6, 10_000_000), (7005, 60, 500, 12, 150_000)]


@pytest.mark.parametrize("seed,B,M,K,R", CASES)
def test_kept_terms_equal_recomputed_and_direct_swaps(orc, seed, B, M, K, R):
    inst = random_instance(seed, B=B, M=M, K=K, clustered=True)
    R = inst.R if R is None else R
    cost = table(orc, inst)
    start, _ = orc.rank(cost, K)
    res = orc.tabu(cost, K, R, 25, 3, start_open=start)
    assert len(res.moves) > 5
    for t, (O, kept, new) in enumerate(replay(orc, cost, K, R, res.moves, start)):
        fresh = terms(cost, *new, R, K)
        cand = np.array([b for b in range(B) if b not in O])
        for q in range(2):
            assert np.array_equal(kept[q][cand], fresh[q][cand]), (t, q)
        for q in (2, 3):
            assert np.array_equal(kept[q][:, cand], fresh[q][:, cand]), (t, q)
        if t % 6 == 0:
            v0c, v0d, lc, ld = loss_v0(*new, R, K)
            fc, fd = orc.swap_table(cost, np.asarray(O, dtype=np.int32), R)
            for k, i in enumerate(O):
                for j in cand:
                    assert (v0c + kept[0][j] + lc[k] + kept[2][k, j],
                            v0d + kept[1][j] + ld[k] + kept[3][k, j]) == (fc[i, j], fd[i, j])


@pytest.mark.parametrize("half", ["rebuild_closed", "take_out_old"])
def test_each_half_of_the_rule_is_needed(orc, half):
    inst = random_instance(7101, B=35, M=800, K=6, clustered=True)
    cost = table(orc, inst)
    start, _ = orc.rank(cost, 6)
    res = orc.tabu(cost, 6, inst.R, 20, 3, start_open=start)
    wrong = False
    for O, kept, new in replay(orc, cost, 6, inst.R, res.moves, start, **{half: False}):
        fresh = terms(cost, *new, inst.R, 6)
        cand = np.array([b for b in range(inst.B) if b not in O])
        if not (np.array_equal(kept[0][cand], fresh[0][cand]) and np.array_equal(kept[3][:, cand],
                                                                              fresh[3][:, cand])):
            wrong = True
            break
    assert wrong
