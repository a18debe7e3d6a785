"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* exact integer arithmetic for the leg distance (Python's isqrt);
* a hand-worked instance (tests/golden/hand_worked_3x2.json);
* closed forms and library routines for special cases (numpy min/sum/argsort);
* brute-force enumeration of every placement on tiny instances;
* invariants (monotone coverage in R, Tabu never worse than its start, never
  better than the optimum, every recorded objective equal to a recomputation);
* an independent brute-force replay of the Tabu rules in Python.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2001_05291_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked_3x2.json")
INF = 2**31 - 1


def exact_ceil_sqrt(n: int) -> int:
    s = math.isqrt(n)
    return s if s * s == n else s + 1


def exact_leg(x1, y1, x2, y2) -> int:
    return exact_ceil_sqrt((x1 - x2) ** 2 + (y1 - y2) ** 2)


def random_instance(rng_seed: int, B=None, M=None, K=None, clustered=None):
    """A small random instance drawn with the synthetic generator."""
    key = synth.stream_key(rng_seed, 99, 0)
    u = synth.u01(synth.draws_u64(key, np.arange(8)))
    B = B or int(3 + u[0] * 12)
    M = M or int(1 + u[1] * 40)
    K = K or int(1 + u[2] * min(5, B - 1))
    K = max(1, min(K, B - 1))
    clustered = bool(u[3] < 0.5) if clustered is None else clustered
    lay = synth.Layout(300_000, 200_000, clustered=clustered, sigma_m=20_000.0)
    R = int(100_000 + u[4] * 900_000)
    return synth.make_instance("rand", rng_seed, B, 2 * B, M, K, R, 30, 3, lay)


def table(orc, inst):
    return orc.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy)


def f_pair(c, R):
    return (1, int(c)) if c <= R else (0, 0)


def F_numpy(cost, open_, R):
    best = cost[np.asarray(open_)].min(axis=0)
    cov = int((best <= R).sum())
    return cov, int(best[best <= R].astype(np.int64).sum())


def better(a, b):
    return a[0] > b[0] or (a[0] == b[0] and a[1] < b[1])


# ---------------------------------------------------------------- leg distance
def test_leg_equals_exact_integer_ceil_sqrt(orc):
    key = synth.stream_key(123, 98, 0)
    u = synth.draws_u64(key, np.arange(40000))
    lim = 2**24
    xs = (u % np.uint64(2 * lim + 1)).astype(np.int64) - lim
    xs = xs.reshape(-1, 4)
    for x1, y1, x2, y2 in xs[:10000]:
        assert orc.leg(int(x1), int(y1), int(x2), int(y2)) == exact_leg(x1, y1, x2, y2)


def test_leg_special_cases(orc):
    # Pythagorean triples: exact squares give exact values
    for (p, q, r) in [(3, 4, 5), (5, 12, 13), (8, 15, 17), (20, 21, 29), (119, 120, 169)]:
        for s in (1, 1000, 99991):
            assert orc.leg(0, 0, p * s, q * s) == r * s
            assert orc.leg(p * s, -q * s, 0, 0) == r * s
    # n = s^2 + 1 (just above a square) and n = s^2 - 1 (just below one)
    for s in (1, 2, 7, 4096, 2**20 + 3, 2**24, 2**25 - 1):
        assert orc.leg(0, 0, s, 1) == s + 1
    for k in (1, 3, 100, 2000, 2895):  # (2k^2)^2 + (2k)^2 = (2k^2+1)^2 - 1
        dx, dy = 2 * k * k, 2 * k
        assert orc.leg(0, 0, dx, dy) == 2 * k * k + 1
    # extremes of the accepted coordinate range |x|, |y| <= 2^24
    lim = 2**24
    assert orc.leg(-lim, -lim, lim, lim) == exact_leg(-lim, -lim, lim, lim)
    assert orc.leg(-lim, 0, lim, 0) == 2**25
    assert orc.leg(5, 5, 5, 5) == 0


def test_cost_table_three_legs(orc):
    inst = random_instance(5, B=7, M=11)
    c = table(orc, inst)
    for b in range(inst.B):
        bx, by = map(int, inst.base_xy[b])
        for m in range(inst.M):
            px, py = map(int, inst.pick_xy[m])
            qx, qy = map(int, inst.drop_xy[m])
            want = exact_leg(bx, by, px, py) + exact_leg(px, py, qx, qy) + exact_leg(qx, qy, bx, by)
            assert c[b, m] == want


# ---------------------------------------------------------------- hand-worked
@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_golden_legs_and_table(orc, golden):
    for leg in golden["legs"]:
        assert orc.leg(*leg["from"], *leg["to"]) == leg["leg"]
    c = orc.cost_table(np.array(golden["base_xy"]), np.array(golden["pick_xy"]),
                       np.array(golden["drop_xy"]))
    assert c.tolist() == golden["cost"]


def test_golden_rank_evaluate_best_two(orc, golden):
    c = np.array(golden["cost"], dtype=np.int32)
    for k, want in golden["rank"].items():
        got, rs = orc.rank(c, int(k[1:]))
        assert got.tolist() == want
        assert rs.tolist() == golden["rowsum"]
    for e in golden["evaluate"]:
        assert orc.evaluate(c, e["open"], e["R"]) == (e["cov"], e["dist"])
    bt = golden["best_two"]
    a, b, b1, b2 = orc.best_two(c, bt["open"])
    assert (a.tolist(), b.tolist(), b1.tolist(), b2.tolist()) == (bt["a"], bt["b"], bt["b1"], bt["b2"])


def test_golden_swaps_and_bruteforce(orc, golden):
    c = np.array(golden["cost"], dtype=np.int32)
    sw = golden["swaps"]
    fc, fd = orc.swap_table(c, sw["open"], sw["R"])
    for e in sw["F"]:
        want = (e["cov"], e["dist"])
        assert (int(fc[e["i"], e["j"]]), int(fd[e["i"], e["j"]])) == want
        assert orc.swap_full(c, sw["open"], sw["R"], e["i"], e["j"]) == want
        assert orc.swap_best_two(c, sw["open"], sw["R"], e["i"], e["j"]) == want
    for e in golden["bruteforce"]:
        o, cov, dist, n = orc.bruteforce(c, e["K"], e["R"])
        assert (sorted(o.tolist()), cov, dist) == (e["open"], e["cov"], e["dist"])
        assert n == math.comb(3, e["K"])


def test_golden_tabu(orc, golden):
    c = np.array(golden["cost"], dtype=np.int32)
    t = golden["tabu"]
    for mode in (0, 1, 2):
        r = orc.tabu(c, t["K"], t["R"], t["iters"], t["tenure"], start_open=t["start"], eval_mode=mode)
        assert [list(m) for m in r.moves] == t["moves"]
        assert r.best_open.tolist() == t["best_open"]
        assert (r.best_cov, r.best_dist, r.best_iter) == (t["best_cov"], t["best_dist"], t["best_iter"])
        assert r.final_open.tolist() == t["final_open"]
    r = orc.tabu(c, t["K"], t["R"], t["iters"], t["tenure"], start_open=t["start"],
                 accept_worsening=False)
    assert [list(m) for m in r.moves] == t["improving_only_moves"]


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("seed", range(6))
def test_evaluate_special_cases(orc, seed):
    inst = random_instance(100 + seed)
    c = table(orc, inst)
    o = np.arange(inst.K)
    best = c[o].min(axis=0)
    # R at least every cost: every mission covered, distance is the K-median objective
    assert orc.evaluate(c, o, INF - 1) == (inst.M, int(best.astype(np.int64).sum()))
    # R below every cost: nothing covered
    assert orc.evaluate(c, o, int(best.min()) - 1) == (0, 0)
    # coverage never decreases as R grows
    prev = -1
    for R in sorted(set(best.tolist())):
        cov, dist = orc.evaluate(c, o, R)
        assert cov >= prev
        assert cov == int((best <= R).sum())
        prev = cov


@pytest.mark.parametrize("seed", range(6))
def test_rank_matches_library_sort(orc, seed):
    inst = random_instance(200 + seed)
    c = table(orc, inst)
    got, rs = orc.rank(c, inst.K)
    S = c.astype(np.int64).sum(axis=1)
    assert rs.tolist() == S.tolist()
    order = np.lexsort((np.arange(inst.B), S))
    assert got.tolist() == order[: inst.K].tolist()
    # with unavailable bases
    avail = np.ones(inst.B, dtype=np.uint8)
    avail[order[0]] = 0
    got2, _ = orc.rank(c, inst.K, avail)
    assert got2.tolist() == [int(x) for x in order if avail[x]][: inst.K]


def with_duplicate_bases(inst, copies=(0, 2, 3)):
    """Bases that repeat earlier bases' coordinates: equal rows, equal row sums,
    equal swap objectives, so every tie-break rule is exercised."""
    extra = inst.base_xy[list(copies)]
    bx = np.concatenate([inst.base_xy, extra, inst.base_xy[:1]], axis=0)
    return synth.Instance(inst.name + "+dup", inst.seed, np.ascontiguousarray(bx), inst.pick_xy,
                          inst.drop_xy, inst.K, inst.R, inst.iters, inst.tenure)


@pytest.mark.parametrize("seed", range(6))
def test_rank_ties_take_lower_index(orc, seed):
    inst = with_duplicate_bases(random_instance(250 + seed, B=8))
    c = table(orc, inst)
    S = c.astype(np.int64).sum(axis=1)
    assert len(set(S.tolist())) < inst.B
    for K in range(1, inst.B):
        got, _ = orc.rank(c, K)
        assert got.tolist() == np.lexsort((np.arange(inst.B), S))[:K].tolist()


@pytest.mark.parametrize("seed", range(12))
def test_tabu_with_ties_matches_bruteforce_replay(orc, seed):
    inst = with_duplicate_bases(random_instance(650 + seed, B=6, M=int(5 + seed)))
    c = table(orc, inst)
    start, _ = orc.rank(c, inst.K)
    moves, best, best_O, best_it = python_tabu(c, inst.K, inst.R, 15, 1 + seed % 3, start)
    r = orc.tabu(c, inst.K, inst.R, 15, 1 + seed % 3)
    assert [tuple(m) for m in r.moves] == moves
    assert r.best_open.tolist() == best_O


@pytest.mark.parametrize("seed", range(6))
def test_rank_top1_is_optimum_when_all_covered(orc, seed):
    """K = 1 and R above every cost: the best single base minimises its row sum."""
    inst = random_instance(300 + seed)
    c = table(orc, inst)
    top, _ = orc.rank(c, 1)
    o, cov, dist, _ = orc.bruteforce(c, 1, INF - 1)
    assert top.tolist() == o.tolist()
    assert (cov, dist) == (inst.M, int(c[o[0]].astype(np.int64).sum()))


# ---------------------------------------------------------------- swap objective
@pytest.mark.parametrize("seed", range(25))
def test_swap_three_ways_agree(orc, seed):
    inst = random_instance(400 + seed)
    c = table(orc, inst)
    K = inst.K
    open_ = np.sort(np.argsort(synth.u01(synth.draws_u64(synth.stream_key(seed, 97), np.arange(inst.B))))[:K])
    avail = np.ones(inst.B, dtype=np.uint8)
    if inst.B - K > 1:
        closed = [b for b in range(inst.B) if b not in set(open_.tolist())]
        avail[closed[0]] = 0
    fc, fd = orc.swap_table(c, open_, inst.R, avail)
    for i in open_:
        for j in range(inst.B):
            if j in open_ or not avail[j]:
                assert fc[i, j] == -1
                continue
            o2 = [j if x == i else x for x in open_]
            want = F_numpy(c, o2, inst.R)
            assert orc.swap_full(c, open_, inst.R, int(i), j) == want
            assert orc.swap_best_two(c, open_, inst.R, int(i), j) == want
            assert (int(fc[i, j]), int(fd[i, j])) == want


def test_best_two_matches_sort(orc):
    for seed in range(10):
        inst = random_instance(500 + seed)
        c = table(orc, inst)
        o = np.arange(inst.B)[::-1][: inst.K].copy()
        a, b, b1, b2 = orc.best_two(c, o)
        for m in range(inst.M):
            keys = sorted((int(c[x, m]), int(x)) for x in o)
            assert (a[m], b1[m]) == keys[0]
            if inst.K > 1:
                assert (b[m], b2[m]) == keys[1]
            else:
                assert (b[m], b2[m]) == (INF, -1)


# ---------------------------------------------------------------- Tabu
def python_tabu(cost, K, R, iters, tenure, start, avail=None, accept_worsening=True):
    """Independent brute-force replay of the Tabu rules (full recomputation of every swap)."""
    B = cost.shape[0]
    avail = np.ones(B, dtype=bool) if avail is None else avail.astype(bool)
    O = list(int(x) for x in start)
    expiry = [0] * B
    cur = F_numpy(cost, O, R)
    best, best_O, best_it = cur, sorted(O), -1
    moves = []
    for t in range(iters):
        cands = []
        for i in O:
            for j in range(B):
                if j in O or not avail[j]:
                    continue
                F = F_numpy(cost, [j if x == i else x for x in O], R)
                tabu = t < expiry[i] or t < expiry[j]
                cands.append(((-F[0], F[1], i, j), F, tabu))
        if not cands:
            break
        adm = [x for x in cands if (not x[2]) or better(x[1], best)]
        flags = 0
        if adm:
            key, F, tabu = min(adm)
            if tabu:
                flags |= 2
        else:
            key, F, tabu = min(cands)
            flags |= 1
        i, j = key[2], key[3]
        if not accept_worsening and not better(F, cur):
            break
        O = [j if x == i else x for x in O]
        expiry[i] = expiry[j] = t + tenure + 1
        cur = F
        if better(F, best):
            best, best_O, best_it = F, sorted(O), t
            flags |= 4
        moves.append((t, i, j, flags, F[0], F[1]))
    return moves, best, best_O, best_it


@pytest.mark.parametrize("seed", range(30))
def test_tabu_matches_bruteforce_replay(orc, seed):
    inst = random_instance(600 + seed, B=int(4 + seed % 7), M=int(3 + (seed * 7) % 25))
    c = table(orc, inst)
    avail = np.ones(inst.B, dtype=np.uint8)
    if seed % 3 == 0 and inst.B - inst.K > 1:
        avail[(seed * 5) % inst.B] = 0
    start, _ = orc.rank(c, inst.K, avail)
    tenure = 1 + seed % 4
    for aw in (True, False):
        moves, best, best_O, best_it = python_tabu(c, inst.K, inst.R, 12, tenure, start, avail, aw)
        r = orc.tabu(c, inst.K, inst.R, 12, tenure, start_open=start, avail=avail, accept_worsening=aw)
        assert [tuple(m) for m in r.moves] == moves
        assert (r.best_cov, r.best_dist) == best
        assert r.best_open.tolist() == best_O
        assert r.best_iter == best_it


@pytest.mark.parametrize("seed,B,M,tenure", [(5031, 10, 17, 2), (5031, 10, 17, 5), (5041, 11, 27, 3),
                                              (5071, 14, 27, 2), (5071, 14, 27, 5)])
def test_tabu_aspiration_matches_bruteforce_replay(orc, seed, B, M, tenure):
    """Instances where a tabu move beats the best so far and is admitted (aspiration)."""
    inst = random_instance(seed, B=B, M=M)
    c = table(orc, inst)
    start, _ = orc.rank(c, inst.K)
    moves, best, best_O, best_it = python_tabu(c, inst.K, inst.R, 20, tenure, start)
    assert any(m[3] & 2 for m in moves)
    r = orc.tabu(c, inst.K, inst.R, 20, tenure)
    assert [tuple(m) for m in r.moves] == moves
    assert (r.best_cov, r.best_dist, r.best_iter) == (best[0], best[1], best_it)


@pytest.mark.parametrize("seed", range(200))
def test_tabu_bounded_by_optimum(orc, seed):
    """Random tiny instances (B <= 22, K <= 6): start <= Tabu best <= brute-force optimum."""
    key = synth.stream_key(seed, 96, 0)
    u = synth.u01(synth.draws_u64(key, np.arange(4)))
    B = int(4 + u[0] * 19)
    K = int(1 + u[1] * min(6, B - 1))
    M = int(5 + u[2] * 40)
    inst = random_instance(700 + seed, B=B, M=M, K=K)
    c = table(orc, inst)
    r = orc.tabu(c, K, inst.R, 25, 3)
    start, _ = orc.rank(c, K)
    s = orc.evaluate(c, start, inst.R)
    best = (r.best_cov, r.best_dist)
    assert not better(s, best)
    _, oc, od, n = orc.bruteforce(c, K, inst.R)
    assert n == math.comb(B, K)
    assert not better(best, (oc, od))
    assert orc.evaluate(c, r.best_open, inst.R) == best
    # every recorded objective is the objective of the placement after the move
    O = list(start)
    for (t, i, j, fl, cov, dist) in r.moves:
        O = [j if x == i else x for x in O]
        assert orc.evaluate(c, O, inst.R) == (cov, dist)
    assert sorted(O) == r.final_open.tolist()


def test_tiny_workload_reaches_optimum(orc):
    """The 20-base tiny workload: Tabu from the ranking reaches the exhaustive optimum."""
    inst = synth.tiny()
    c = table(orc, inst)
    o, cov, dist, n = orc.bruteforce(c, inst.K, inst.R)
    assert n == 15504
    r = orc.tabu(c, inst.K, inst.R, inst.iters, inst.tenure)
    assert (r.best_cov, r.best_dist) == (cov, dist)


@pytest.mark.parametrize("seed", range(5))
def test_bruteforce_optimum_monotone_in_R(orc, seed):
    inst = random_instance(800 + seed, B=9, M=25, K=3)
    c = table(orc, inst)
    prev = -1
    for R in np.linspace(int(c.min()) - 1, int(c.max()), 12).astype(int):
        _, cov, _, _ = orc.bruteforce(c, 3, int(R))
        assert cov >= prev
        prev = cov


def test_tabu_resume_equals_uninterrupted(orc):
    inst = synth.tiny()
    c = table(orc, inst)
    full = orc.tabu(c, inst.K, inst.R, 40, inst.tenure)
    first = orc.tabu(c, inst.K, inst.R, 15, inst.tenure)
    # the final placement of the first leg, in the oracle's own slot order, is a set
    second = orc.tabu(c, inst.K, inst.R, 25, inst.tenure, start_open=first.final_open, t0=15,
                      expiry_in=first.expiry, best_in=first.best_open, best_cov_in=first.best_cov,
                      best_dist_in=first.best_dist, best_iter_in=first.best_iter)
    assert [tuple(m) for m in first.moves + second.moves] == [tuple(m) for m in full.moves]
    assert (second.best_cov, second.best_dist, second.best_iter) == (full.best_cov, full.best_dist, full.best_iter)
    assert second.best_open.tolist() == full.best_open.tolist()


def test_improving_only_stops_at_local_optimum(orc):
    """The paper's rule (Sec. 4.3): only improving moves; at the end no swap improves."""
    for seed in range(8):
        inst = random_instance(900 + seed, B=12, M=30, K=3)
        c = table(orc, inst)
        r = orc.tabu(c, 3, inst.R, 200, 0, accept_worsening=False)
        cur = (r.final_cov, r.final_dist)
        fc, fd = orc.swap_table(c, r.final_open, inst.R)
        for i in r.final_open:
            for j in range(inst.B):
                if fc[i, j] >= 0:
                    assert not better((int(fc[i, j]), int(fd[i, j])), cur)
        assert len(r.moves) < 200


def test_ranking_beats_random_mean(orc):
    """Sec. 5: base ranking starts better than the mean of 100 random placements
    (total distance, every mission counted).  Checked on uniform layouts only: on
    clustered layouts the K bases with the smallest row sums crowd into one
    cluster and the claim does not hold (the province workload is an example)."""
    for inst in (synth.tiny(), random_instance(1000, B=40, M=300, K=6, clustered=False)):
        c = table(orc, inst)
        start, _ = orc.rank(c, inst.K)
        Rall = INF - 1
        s = orc.evaluate(c, start, Rall)[1]
        key = synth.stream_key(inst.seed, 95, 0)
        tot = 0
        for r in range(100):
            u = synth.u01(synth.draws_u64(key, np.arange(inst.B) + r * inst.B))
            pick = np.argsort(u)[: inst.K]
            tot += orc.evaluate(c, pick, Rall)[1]
        assert s < tot / 100
