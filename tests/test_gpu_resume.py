"""Batch requests that resume from the resident instance's kept state
(stage_request.resume_resident), against the oracle given the same state.

* Without an update in between, a resumed request continues the search:
  first + second = one uninterrupted oracle search.
* After an update (missions added and removed, open bases made unavailable)
  the open bases the update closed leave by forced moves (reading A15), the
  best so far restarts from the resumed placement, and the search continues
  with the kept tabu expiries and iteration number: equal to the oracle's
  forced moves followed by its search from that state.
* The same request among other requests in one batch gives the same result.
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


def small(seed, B, M, K, R=350_000):
    lay = synth.Layout(400_000, 300_000, clustered=True, sigma_m=25_000.0)
    return synth.make_instance(f"r{seed}", seed, B, 2 * B, M, K, R, 20, 4, lay)


def moves(res):
    return [tuple(int(x) for x in m) for m in res.moves]


def run_scenario(stage, mix, **ctx_kwargs):
    inst = small(31, 90, 5000, 6)
    extra = small(32, 90, 400, 6)
    K, R, tenure = inst.K, inst.R, 4
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    o1 = oracle.tabu(cost, K, R, 20, tenure, nthreads=8)
    o2 = oracle.tabu(cost, K, R, 15, tenure, start_open=o1.final_open, t0=20, expiry_in=o1.expiry,
                     best_in=o1.best_open, best_cov_in=o1.best_cov, best_dist_in=o1.best_dist,
                     best_iter_in=o1.best_iter, nthreads=8)
    # the update: two of the open bases close, missions come and go
    gone = [int(o2.final_open[0]), int(o2.final_open[3])]
    remove = np.arange(0, inst.M, 9)
    pick = np.concatenate([inst.pick_xy, extra.pick_xy])
    drop = np.concatenate([inst.drop_xy, extra.drop_xy])
    keep = np.ones(len(pick), bool)
    keep[remove] = False
    cost3 = oracle.cost_table(inst.base_xy, pick[keep], drop[keep], 8)
    avail = np.ones(inst.B, np.uint8)
    avail[gone] = 0
    O3, exp3, done = oracle.forced_moves(cost3, list(o2.final_open), R, avail, 35, tenure, o2.expiry)
    cov3, dist3 = oracle.evaluate(cost3, O3, R)
    o3 = oracle.tabu(cost3, K, R, 25, tenure, start_open=O3, avail=avail, t0=35, expiry_in=exp3, best_in=O3,
                     best_cov_in=cov3, best_dist_in=dist3, best_iter_in=-1, nthreads=8)
    assert len(done) == 2
    with stage.Context(device=0, max_slots=8, **ctx_kwargs) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        base = dict(inst=h, K=K, R=R, tenure=tenure, resume_resident=True)
        r1 = ctx.batch_submit([dict(base, iters=20)])[0].wait()
        r2 = ctx.batch_submit([dict(base, iters=15)])[0].wait()
        req3 = dict(base, iters=25, update=dict(add_pick=extra.pick_xy, add_drop=extra.drop_xy, remove=remove,
                                                unavailable=gone))
        others = []
        if mix:
            for s in range(5):
                o = small(40 + s, 40 + 10 * s, 2000 + 500 * s, 4)
                others.append((o, dict(base_xy=o.base_xy, pick_xy=o.pick_xy, drop_xy=o.drop_xy, K=o.K, R=o.R,
                                       iters=15, tenure=3)))
        tickets = ctx.batch_submit([req3] + [rq for _, rq in others])
        r3 = tickets[0].wait()
        rest = [t.wait() for t in tickets[1:]]
    assert moves(r1) == [tuple(m) for m in o1.moves]
    assert r1.n_forced == 0 and r2.n_forced == 0
    assert moves(r2) == [tuple(m) for m in o2.moves]
    assert (r2.best_cov, r2.best_dist, r2.best_iter) == (o2.best_cov, o2.best_dist, o2.best_iter)
    assert r3.n_forced == 2
    assert moves(r3) == [tuple(m) for m in o3.moves]
    assert (r3.best_cov, r3.best_dist, r3.best_iter) == (o3.best_cov, o3.best_dist, o3.best_iter)
    assert np.array_equal(np.sort(r3.final_open), o3.final_open)
    for (o, _), got in zip(others, rest):
        want = oracle.tabu(oracle.cost_table(o.base_xy, o.pick_xy, o.drop_xy, 8), o.K, o.R, 15, 3, nthreads=8)
        assert moves(got) == [tuple(m) for m in want.moves]


def test_resumed_requests_alone(stage_mod):
    run_scenario(stage_mod, mix=False)


def test_resumed_requests_in_a_mix(stage_mod):
    run_scenario(stage_mod, mix=True)


def test_resumed_requests_grouped_incremental_slots(stage_mod):
    run_scenario(stage_mod, mix=True, incremental=True, persist=False)


def test_resumed_requests_grouped_full_pass_slots(stage_mod):
    run_scenario(stage_mod, mix=True, persist=False)


def test_resume_without_resident_state_starts_from_the_ranking(stage_mod):
    inst = small(33, 50, 3000, 5)
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    want = oracle.tabu(cost, inst.K, inst.R, 12, 3, nthreads=8)
    with stage_mod.Context(device=0) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        # a request without the flag keeps nothing
        ctx.batch_submit([dict(inst=h, K=inst.K, R=inst.R, iters=12, tenure=3)])[0].wait()
        got = ctx.batch_submit([dict(inst=h, K=inst.K, R=inst.R, iters=12, tenure=3,
                                     resume_resident=True)])[0].wait()
        # another K: the kept state (K = 5) does not apply
        other = ctx.batch_submit([dict(inst=h, K=4, R=inst.R, iters=12, tenure=3,
                                       resume_resident=True)])[0].wait()
    assert moves(got) == [tuple(m) for m in want.moves] and got.n_forced == 0
    w4 = oracle.tabu(cost, 4, inst.R, 12, 3, nthreads=8)
    assert moves(other) == [tuple(m) for m in w4.moves]
