"""The placement of stage_tabu_batch's searches on the GPU's CTAs (host logic,
no device): every search gets its gang of distinct CTAs, every CTA runs its
searches in one global order, and so a simulation of the CTAs -- each running
its entries in order, a search starting once all of its CTAs have reached it
-- always finishes every search (the gang barriers cannot deadlock), at the
estimated makespan; on the batched workload's shapes that makespan is within
1.2 times the larger lower bound (the busiest search, the work over the CTAs).
"""
import itertools

import numpy as np
import pytest

from paper_2001_05291_gb300 import build, stage


@pytest.fixture(scope="module")
def sched():
    build.build()
    return stage.batch_schedule


def simulate(lists, us, gang):
    """Each CTA runs its entries in order; search k starts when all gang[k] of
    its CTAs have arrived and ends us[k] later.  Returns (finished searches,
    makespan); a deadlock leaves searches unfinished."""
    P = len(lists)
    pos, t = [0] * P, [0.0] * P
    arrived, done = {}, set()
    moved = True
    while moved:
        moved = False
        for q in range(P):
            if pos[q] >= len(lists[q]):
                continue
            k, _ = lists[q][pos[q]]
            arr = arrived.setdefault(k, {})
            if q not in arr:
                arr[q] = t[q]
                moved = True
            if len(arr) == gang[k] and k not in done:
                end = max(arr.values()) + us[k]
                for qq in arr:
                    t[qq] = end
                    pos[qq] += 1
                done.add(k)
                moved = True
    return done, max(t) if P else 0.0


def check(sched, us, gang, P):
    lists, mk = sched(us, gang, P)
    n = len(us)
    # each search: gang[k] entries, ranks 0..g-1, on distinct CTAs
    seen = {}
    for q, lst in enumerate(lists):
        for k, r in lst:
            seen.setdefault(k, []).append((q, r))
    assert sorted(seen) == list(range(n))
    for k, ent in seen.items():
        assert len(ent) == gang[k]
        assert sorted(r for _, r in ent) == list(range(gang[k]))
        assert len({q for q, _ in ent}) == gang[k]
    # one global order: any two searches sharing CTAs are met in the same
    # order on all of them
    rank_on = [{k: i for i, (k, _) in enumerate(lst)} for lst in lists]
    for a, b in itertools.combinations(range(n), 2):
        shared = [q for q in range(P) if a in rank_on[q] and b in rank_on[q]]
        assert len({rank_on[q][a] < rank_on[q][b] for q in shared}) <= 1
    done, sim = simulate(lists, us, gang)
    assert len(done) == n, "a gang barrier would never be passed"
    assert sim == pytest.approx(mk, rel=1e-12, abs=1e-9)
    area = float(np.dot(us, gang)) / P
    longest = float(max(us)) if n else 0.0
    assert mk >= max(area, longest) - 1e-9
    return mk, area, longest


def test_random_batches(sched):
    """Correctness on uneven draws (gangs up to 16 on 1 to 39 CTAs).  No
    quality bound is asserted here: gangs wide against P leave holes that no
    list schedule of rigid gangs avoids in general."""
    rng = np.random.default_rng(7)
    for trial in range(60):
        P = int(rng.integers(1, 40))
        n = int(rng.integers(0, 80))
        gang = np.minimum(2 ** rng.integers(0, 5, n), P).astype(np.int32)
        us = np.exp(rng.uniform(0, 6, n))
        check(sched, us, gang, P)


def test_gangs_that_overlap_in_a_cycle(sched):
    """Three searches pairwise sharing a CTA (an order that differs between
    CTAs would deadlock), and equal times (ties broken by index)."""
    check(sched, [5.0, 5.0, 5.0], [2, 2, 2], 3)
    check(sched, [3.0, 2.0, 1.0, 4.0], [3, 1, 2, 2], 3)


def test_batched_workload_shapes(sched):
    """512 searches as the batched workload's gang rule sizes them, on 152 CTAs."""
    rng = np.random.default_rng(3)
    us = np.exp(rng.uniform(np.log(300.0), np.log(4e6), 512))
    ideal = us.sum() / 152
    gang = np.ones(512, dtype=np.int32)
    for k in range(512):
        while gang[k] * 2 <= 128 and us[k] / gang[k] > 0.5 * ideal:
            gang[k] *= 2
    mk, area, longest = check(sched, us / gang, gang, 152)
    assert mk <= 1.2 * max(area, longest)   # about 1.13-1.16 on such draws


def test_refused_arguments(sched):
    with pytest.raises(stage.StageError):
        sched([1.0, 2.0], [1, 0], 4)
    with pytest.raises(stage.StageError):
        sched([1.0], [5], 4)
    assert sched([], [], 3)[0] == [[], [], []]
