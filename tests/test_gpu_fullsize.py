"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle cannot run 1000 iterations on an 8 GB table in a test, so the checks
are: the first moves against the oracle's own search on the full table (the
trajectory of a longer run starts with the shorter run's); sampled later moves
against the move the oracle takes from the state (placement, tabu expiries,
best so far) that the GPU's earlier moves lead to; and the best placement and
sampled placements against the oracle's evaluation.  All quantities are
integers: zero tolerance.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2001_05291_gb300 import synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def stage_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage
    build.build()
    return stage


def replay(start, moves):
    """Placements after each move, from the start placement."""
    O = [int(x) for x in start]
    out = []
    for (_, i, j, *_r) in moves:
        O = [j if x == i else x for x in O]
        out.append(list(O))
    return out


def state_before(cost, R, start, moves, t, tenure):
    """The search state before move t, rebuilt from the GPU's trajectory: the
    placement, the tabu expiries (both bases of a move at iteration u stay tabu
    until u + tenure + 1) and the best so far (changed only by a strictly better
    placement; the start's iteration is -1)."""
    O = [int(x) for x in start]
    expiry = np.zeros(cost.shape[0], dtype=np.int32)
    best = oracle.evaluate(cost, O, R)
    best_open, best_iter = list(O), -1
    for (it, i, j, _f, cov, dist) in moves[:t]:
        O = [j if x == i else x for x in O]
        expiry[i] = expiry[j] = it + tenure + 1
        if cov > best[0] or (cov == best[0] and dist < best[1]):
            best, best_open, best_iter = (cov, dist), list(O), it
    return O, expiry, best, best_open, best_iter


def check_sampled_moves(cost, K, R, tenure, start, moves, samples):
    """Each sampled GPU move t is the move the oracle takes from the state the
    GPU's first t moves lead to: the best admissible swap of the whole
    neighbourhood under the tabu, aspiration, fallback and tie rules, with its
    flags and objective."""
    for t in samples:
        O, expiry, best, best_open, best_iter = state_before(cost, R, start, moves, t, tenure)
        ref = oracle.tabu(cost, K, R, 1, tenure, start_open=O, nthreads=THREADS, t0=moves[t][0], expiry_in=expiry,
                          best_in=best_open, best_cov_in=best[0], best_dist_in=best[1], best_iter_in=best_iter)
        assert [tuple(m) for m in ref.moves] == [tuple(moves[t])], f"move {t}"


def test_large_workload_as_benchmarked(stage_mod):
    stage = stage_mod
    inst = synth.large()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, THREADS)
    with stage.Context(device=0) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        start, rowsum = ctx.rank_bases(h, inst.K, inst.B)
        got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
        # sampled table windows (caller's mission order) against the oracle's table
        key = synth.stream_key(2, 90)
        u = synth.draws_u64(key, np.arange(64))
        for k in range(0, 64, 2):
            b, m = int(u[k] % np.uint64(inst.B - 4)), int(u[k + 1] % np.uint64(inst.M - 512))
            assert np.array_equal(ctx.read_table(h, b, 4, m, 512), cost[b:b + 4, m:m + 512])
    assert got.n_moves == inst.iters
    wo, wrs = oracle.rank(cost, inst.K)
    assert np.array_equal(start, wo) and np.array_equal(rowsum, wrs)
    ref = oracle.tabu(cost, inst.K, inst.R, 2, inst.tenure, nthreads=THREADS)
    assert [tuple(m) for m in got.moves[:2]] == [tuple(m) for m in ref.moves]
    placements = replay(start, got.moves)
    for t in (2, 100, 500, inst.iters - 1):
        assert oracle.evaluate(cost, placements[t], inst.R) == (got.moves[t][4], got.moves[t][5])
    assert oracle.evaluate(cost, got.best_open, inst.R) == (got.best_cov, got.best_dist)
    assert sorted(placements[-1]) == got.final_open.tolist()
    # later moves: each one the oracle's choice from the state the GPU reached
    check_sampled_moves(cost, inst.K, inst.R, inst.tenure, start, got.moves, (2, 100, 500, inst.iters - 1))
    # the search as benchmarked keeps the neighbourhood's terms across
    # iterations; re-evaluating the whole table every iteration gives the same
    # 1000 moves
    with stage.Context(device=0, full_pass=True) as cf:
        hf = cf.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        full = cf.tabu_run(hf, inst.K, inst.R, inst.iters, inst.tenure)
        cf.unload_instance(hf)
    assert [tuple(m) for m in full.moves] == [tuple(m) for m in got.moves]
    assert (full.best_cov, full.best_dist, full.best_iter) == (got.best_cov, got.best_dist, got.best_iter)


def test_batched_workload_instances_in_one_batch(stage_mod):
    stage = stage_mod
    sizes = synth.batched_sizes()
    # the largest, the smallest and a spread of the 512 instances, at their full sizes
    order = np.argsort([(B - K) * M for B, M, K, R in sizes])
    pick = [int(order[-1]), int(order[0]), int(order[128]), int(order[256]), int(order[384]), int(order[500])]
    insts = [synth.batched_instance(3, k, *sizes[k]) for k in pick]
    with stage.Context(device=0, max_slots=512) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
        res = [t.wait() for t in ctx.batch_submit(
            [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)])]
        starts = [ctx.rank_bases(h, i.K)[0] for h, i in zip(hs, insts)]
    for inst, r, start in zip(insts, res, starts):
        assert r.n_moves == inst.iters
        cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, THREADS)
        ref = oracle.tabu(cost, inst.K, inst.R, 12, inst.tenure, nthreads=THREADS)
        assert [tuple(m) for m in r.moves[:12]] == [tuple(m) for m in ref.moves]
        placements = replay(start, r.moves)
        for t in (50, inst.iters - 1):
            assert oracle.evaluate(cost, placements[t], inst.R) == (r.moves[t][4], r.moves[t][5])
        assert oracle.evaluate(cost, r.best_open, inst.R) == (r.best_cov, r.best_dist)
        check_sampled_moves(cost, inst.K, inst.R, inst.tenure, start, r.moves, (50, 150, inst.iters - 1))


def test_batched_workload_in_one_launch(stage_mod):
    """All 512 searches of the batched workload in one stage_tabu_batch launch,
    as bench.py times it (the second call, its gangs sized from the first's
    measured costs): every result equals the batch engine's (itself equal to
    each search alone), and six instances across the size range are checked
    against the oracle as above."""
    stage = stage_mod
    insts = synth.batched()
    sizes = synth.batched_sizes()
    order = np.argsort([(B - K) * M for B, M, K, R in sizes])
    pick = [int(order[-1]), int(order[0]), int(order[128]), int(order[256]), int(order[384]), int(order[500])]
    with stage.Context(device=0, max_slots=512) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
        reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
        first = ctx.tabu_batch(reqs)
        res = ctx.tabu_batch(reqs)
        assert ctx.kernel_stats("batch_gang_max")[0] > 1
        eng = [t.wait() for t in ctx.batch_submit(reqs)]
        starts = {k: ctx.rank_bases(hs[k], insts[k].K)[0] for k in pick}
    for a, b, c in zip(res, first, eng):
        assert a.moves == b.moves == c.moves
        assert (a.best_cov, a.best_dist, a.best_iter) == (c.best_cov, c.best_dist, c.best_iter)
        assert np.array_equal(np.sort(a.best_open), np.sort(c.best_open))
    for k in pick:
        inst, r, start = insts[k], res[k], starts[k]
        assert r.n_moves == inst.iters
        cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, THREADS)
        ref = oracle.tabu(cost, inst.K, inst.R, 12, inst.tenure, nthreads=THREADS)
        assert [tuple(m) for m in r.moves[:12]] == [tuple(m) for m in ref.moves]
        placements = replay(start, r.moves)
        assert oracle.evaluate(cost, placements[inst.iters - 1], inst.R) == (r.moves[-1][4], r.moves[-1][5])
        assert oracle.evaluate(cost, r.best_open, inst.R) == (r.best_cov, r.best_dist)
        check_sampled_moves(cost, inst.K, inst.R, inst.tenure, start, r.moves, (100, inst.iters - 1))


def test_local_search_large_workload(stage_mod):
    """Local search (Alg. 2) on the large workload: the first moves equal the
    oracle's on the full table; the complete run's sampled placements, final
    objective and strict improvement are checked against the oracle's
    evaluation."""
    stage = stage_mod
    inst = synth.large()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, THREADS)
    ps, pc = synth.scan_orders(inst.seed, 16, inst.K, inst.B - inst.K)
    with stage.Context(device=0) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        start, _ = ctx.rank_bases(h, inst.K, inst.B)
        first = ctx.local_search(h, inst.K, inst.R, ps, pc, max_moves=3)
        full = ctx.local_search(h, inst.K, inst.R, ps, pc)
    ref = oracle.local_search(cost, inst.K, inst.R, ps, pc, max_moves=3, nthreads=THREADS)
    assert [tuple(m) for m in first.moves] == [tuple(m) for m in ref.moves]
    assert [tuple(m) for m in full.moves[:3]] == [tuple(m) for m in ref.moves]
    placements = replay(start, full.moves)
    covs = [(m[4], -m[5]) for m in full.moves]
    assert all(a < b for a, b in zip(covs, covs[1:]))
    for t in sorted({0, len(placements) // 2, len(placements) - 1}):
        assert oracle.evaluate(cost, placements[t], inst.R) == (full.moves[t][4], full.moves[t][5])
    assert oracle.evaluate(cost, full.final_open, inst.R) == (full.final_cov, full.final_dist)
