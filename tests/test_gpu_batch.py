"""Batch engine and instance updates on the GPU, against runs alone and the oracle.

Every search in a batch must be exactly the search stage_tabu_run performs
alone, whatever else shares the GPU (integers: zero tolerance), and an updated
instance must behave exactly like an instance built from scratch with the
updated mission list (removed missions are INT32_MAX tombstones, appended
missions take the next ids).
"""
import numpy as np
import pytest

import oracle
from paper_2001_05291_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stage_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage
    build.build()
    return stage


def small(seed, B, M, K, R=350_000, iters=30, tenure=4):
    lay = synth.Layout(400_000, 300_000, clustered=True, sigma_m=25_000.0)
    return synth.make_instance(f"b{seed}", seed, B, 2 * B, M, K, R, iters, tenure, lay)


def table(inst):
    return oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)


def same(got, want):
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist, want.best_iter)
    assert np.array_equal(np.sort(got.best_open), np.sort(want.best_open))
    assert np.array_equal(np.sort(got.final_open), np.sort(want.final_open))


MODES = {   # engine modes: Context keyword arguments
    "persistent": dict(),                                    # slots advanced by the persistent batch launch
    "grouped": dict(persist=False),                          # grouped launches, a full pass per step below 8 MB
    "grouped-incremental": dict(persist=False, incremental=True),   # grouped launches, terms kept across steps
}


@pytest.mark.parametrize("mode", list(MODES))
def test_batch_equals_alone_and_oracle(stage_mod, mode):
    """Every slot's search equals its solo run and the oracle, whichever way
    the engine advances it: the persistent batch launch (the slot's terms kept
    across steps inside it), grouped launches with a full pass per step, or
    grouped launches keeping the terms (one full pass, then the records of the
    missions each move touched)."""
    stage = stage_mod
    insts = [small(s, B, M, K, R=R, iters=it) for s, (B, M, K, R, it) in enumerate(
        [(30, 2000, 4, 300_000, 30), (55, 17000, 9, 350_000, 25), (12, 300, 11, 250_000, 20),
         (80, 33000, 16, 400_000, 15), (40, 5000, 6, 200_000, 40), (9, 64, 3, 500_000, 12),
         (70, 20000, 32, 350_000, 18), (25, 9000, 5, 150_000, 35)])]
    with stage.Context(device=0, max_slots=3, profile=True, **MODES[mode]) as ctx:   # queueing
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
        reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
        # an instance given by value, an explicit start, an improving-only search
        v = small(99, 33, 4000, 5)
        reqs.append(dict(base_xy=v.base_xy, pick_xy=v.pick_xy, drop_xy=v.drop_xy, K=5, R=v.R, iters=25,
                         tenure=3))
        reqs.append(dict(inst=hs[1], K=9, R=insts[1].R, iters=20, tenure=2, start_open=np.arange(9)))
        reqs.append(dict(inst=hs[3], K=16, R=insts[3].R, iters=60, tenure=0, accept_worsening=False))
        tickets = ctx.batch_submit(reqs)
        got = [t.wait() for t in tickets]
        for k, (rq, g) in enumerate(zip(reqs, got)):
            if "inst" in rq:
                idx = hs.index(rq["inst"])
                src = insts[idx]
                alone = ctx.tabu_run(rq["inst"], rq["K"], rq["R"], rq["iters"], rq["tenure"],
                                     start_open=rq.get("start_open"),
                                     accept_worsening=rq.get("accept_worsening", True))
                same(g, alone)
            else:
                src = v
            want = oracle.tabu(table(src), rq["K"], rq["R"], rq["iters"], rq["tenure"],
                               start_open=rq.get("start_open"), accept_worsening=rq.get("accept_worsening", True),
                               nthreads=8)
            same(g, want)
            assert g.timing["submit_ns"] <= g.timing["start_ns"] <= g.timing["end_ns"]
        if mode == "grouped-incremental":
            assert ctx.kernel_stats("group_delta")[0] > 0
        if mode == "persistent":
            assert ctx.kernel_stats("engine_persist")[0] > 0
        assert got[-1].n_moves < 60   # the improving-only search stopped early inside the batch


@pytest.mark.parametrize("incremental", [False, True])
def test_update_matches_rebuilt_instance(stage_mod, incremental):
    """An updated instance searches like the rebuilt one; with the incremental
    neighbourhood the search before the update builds the mission-major copy,
    the one after it (more missions, some removed) rebuilds it."""
    stage = stage_mod
    inst = small(7, 45, 12000, 7)
    key = synth.stream_key(7, 50)
    u = synth.u01(synth.draws_u64(key, np.arange(3000)))
    remove = np.unique((u[:400] * inst.M).astype(np.int64))
    add = synth.make_instance("add", 8, 1, 80, 500, 1, 0, 0, 0, synth.Layout(400_000, 300_000))
    closed = [2, 11, 30]
    with stage.Context(device=0, incremental=incremental) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        if incremental:
            before = ctx.tabu_run(h, inst.K, inst.R, 30, 4)
            same(before, oracle.tabu(table(inst), inst.K, inst.R, 30, 4, nthreads=8))
        ctx.update_instance(h, add_pick=add.pick_xy, add_drop=add.drop_xy, remove=remove, unavailable=closed)
        keep = np.setdiff1d(np.arange(inst.M), remove)
        pick = np.concatenate([inst.pick_xy[keep], add.pick_xy])
        drop = np.concatenate([inst.drop_xy[keep], add.drop_xy])
        avail = np.ones(inst.B, dtype=np.uint8)
        avail[closed] = 0
        cost = oracle.cost_table(inst.base_xy, pick, drop, 8)
        # the table by caller ids: removed ids read as INT32_MAX, appended ids follow the originals
        M1 = inst.M + add.M
        got_t = ctx.read_table(h, 0, inst.B, 0, M1)
        want_t = np.full((inst.B, M1), 2**31 - 1, dtype=np.int32)
        want_t[:, keep] = cost[:, : keep.size]
        want_t[:, inst.M:] = cost[:, keep.size:]
        assert np.array_equal(got_t, want_t)
        o, rs = ctx.rank_bases(h, inst.K, inst.B)
        wo, wrs = oracle.rank(cost, inst.K, avail)
        assert np.array_equal(o, wo) and np.array_equal(rs, wrs)
        got = ctx.tabu_run(h, inst.K, inst.R, 40, 4)
        want = oracle.tabu(cost, inst.K, inst.R, 40, 4, avail=avail, nthreads=8)
        same(got, want)
        # reopen a base, remove again (idempotent for already removed ids)
        ctx.update_instance(h, remove=remove[:10], available=[11])
        avail[11] = 1
        got = ctx.tabu_run(h, inst.K, inst.R, 20, 3)
        want = oracle.tabu(cost, inst.K, inst.R, 20, 3, avail=avail, nthreads=8)
        same(got, want)


def test_batch_updates_run_in_order(stage_mod):
    stage = stage_mod
    inst = small(17, 30, 6000, 5)
    with stage.Context(device=0, max_slots=4) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        rm = np.arange(0, 6000, 7)
        t = ctx.batch_submit([dict(inst=h, K=5, R=inst.R, iters=20, tenure=3),
                              dict(inst=h, K=5, R=inst.R, iters=20, tenure=3,
                                   update=dict(remove=rm, unavailable=[1, 4]))])
        first, second = t[0].wait(), t[1].wait()
        cost = table(inst)
        same(first, oracle.tabu(cost, 5, inst.R, 20, 3, nthreads=8))
        keep = np.setdiff1d(np.arange(6000), rm)
        avail = np.ones(30, dtype=np.uint8)
        avail[[1, 4]] = 0
        same(second, oracle.tabu(cost[:, keep], 5, inst.R, 20, 3, avail=avail, nthreads=8))


def test_batch_admission_and_errors(stage_mod):
    stage = stage_mod
    big = small(23, 60, 40000, 6)      # ~10 MB table
    tiny = small(24, 10, 200, 3)
    with stage.Context(device=0, hbm_budget=4 << 20) as ctx:
        t = ctx.batch_submit([dict(base_xy=big.base_xy, pick_xy=big.pick_xy, drop_xy=big.drop_xy, K=6,
                                   R=big.R, iters=5, tenure=2),
                              dict(base_xy=tiny.base_xy, pick_xy=tiny.pick_xy, drop_xy=tiny.drop_xy, K=3,
                                   R=tiny.R, iters=5, tenure=2)])
        with pytest.raises(stage.StageError) as e:
            t[0].wait()
        assert e.value.status == -4            # can never fit the budget
        r = t[1].wait()
        same(r, oracle.tabu(table(tiny), 3, tiny.R, 5, 2))
        with pytest.raises(stage.StageError) as e:
            ctx.batch_submit([dict(base_xy=tiny.base_xy, pick_xy=tiny.pick_xy, drop_xy=tiny.drop_xy, K=300,
                                   R=tiny.R, iters=5, tenure=2)])[0].wait()
        assert e.value.status == -1


def test_requests_on_one_instance_keep_their_order(stage_mod):
    """Each removal names a mission the request just before it added: out of
    order, the removal would be refused (an unknown id).  Requests arrive one
    by one with other traffic between them, so releases of waiting requests
    and admissions of new ones interleave."""
    stage = stage_mod
    inst = small(51, 40, 2000, 4)
    with stage.Context(device=0, max_slots=6) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        n_ids, tickets = inst.M, []
        for k in range(48):
            if k % 2 == 0:
                add = small(60 + k, 40, 30, 4)
                upd = dict(add_pick=add.pick_xy, add_drop=add.drop_xy)
                n_ids += 30
            else:
                upd = dict(remove=[n_ids - 1 - (k % 30)])
            tickets += ctx.batch_submit([dict(inst=h, K=4, R=inst.R, iters=3, tenure=2, update=upd,
                                              resume_resident=(k % 3 == 0))])
            other = small(200 + k, 30, 1500, 3)
            tickets += ctx.batch_submit([dict(base_xy=other.base_xy, pick_xy=other.pick_xy, drop_xy=other.drop_xy,
                                              K=3, R=other.R, iters=3, tenure=2)])
        for t in tickets:
            t.wait()   # raises on a refused request
