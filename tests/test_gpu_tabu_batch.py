"""Many Tabu searches in one persistent launch (stage_tabu_batch), against each
search run alone and the oracle.

Every search of the batch must be exactly the search stage_tabu_run performs
alone (integers: zero tolerance), whatever gang of CTAs it ran on and whatever
else shared the launch.
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
    return synth.make_instance(f"tb{seed}", seed, B, 2 * B, M, K, R, iters, tenure, lay)


def same(got, want):
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist, want.best_iter)
    assert np.array_equal(np.sort(got.best_open), np.sort(want.best_open))
    assert np.array_equal(np.sort(got.final_open), np.sort(want.final_open))


SHAPES = [  # B, M, K, R, iters
    (30, 2000, 4, 300_000, 30), (55, 17000, 9, 350_000, 25), (12, 300, 11, 250_000, 20),
    (80, 33000, 16, 400_000, 15), (40, 5000, 6, 200_000, 40), (9, 64, 3, 500_000, 12),
    (70, 20000, 32, 350_000, 18), (25, 9000, 5, 150_000, 35), (300, 1000, 1, 300_000, 20),
    (64, 777, 12, 10**9, 10),
]


def test_one_launch_equals_alone_and_oracle(stage_mod):
    """Uneven shapes, K = 1, R beyond every cost, an explicit start, the
    improving-only rule, unavailable bases, a search with no candidate and
    one with no iteration, all in one call."""
    stage = stage_mod
    insts = [small(s, B, M, K, R=R, iters=it) for s, (B, M, K, R, it) in enumerate(SHAPES)]
    avail = np.ones(insts[3].B, dtype=np.uint8)
    avail[[2, 17, 40]] = 0
    full = small(50, 9, 500, 9)        # K = B: no closed base to open
    none = small(51, 20, 800, 4)       # iters = 0
    with stage.Context(device=0, profile=True) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy,
                                base_available=avail if k == 3 else None) for k, i in enumerate(insts)]
        reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
        reqs[1]["start_open"] = np.arange(9)
        reqs[4].update(tenure=0, accept_worsening=False, iters=60)
        hf = ctx.load_instance(full.base_xy, full.pick_xy, full.drop_xy)
        hn = ctx.load_instance(none.base_xy, none.pick_xy, none.drop_xy)
        reqs.append(dict(inst=hf, K=9, R=full.R, iters=10, tenure=2))
        reqs.append(dict(inst=hn, K=4, R=none.R, iters=0, tenure=2))
        srcs = insts + [full, none]
        got = ctx.tabu_batch(reqs)
        assert ctx.kernel_stats("tabu_batch")[0] == 1
        assert ctx.kernel_stats("batch_searches")[0] == len(insts)
        for k, (rq, g, src) in enumerate(zip(reqs, got, srcs)):
            alone = ctx.tabu_run(rq["inst"], rq["K"], rq["R"], rq["iters"], rq["tenure"],
                                 start_open=rq.get("start_open"),
                                 accept_worsening=rq.get("accept_worsening", True))
            same(g, alone)
            cost = oracle.cost_table(src.base_xy, src.pick_xy, src.drop_xy, 8)
            want = oracle.tabu(cost, rq["K"], rq["R"], rq["iters"], rq["tenure"],
                               start_open=rq.get("start_open"), avail=avail if k == 3 else None,
                               accept_worsening=rq.get("accept_worsening", True), nthreads=8)
            same(g, want)
        assert got[-2].n_moves == 0 and got[-1].n_moves == 0


def test_gangs_and_repeated_calls(stage_mod):
    """A search large enough to span several CTAs beside many small ones; the
    same call twice gives the same results (the scratch is reused)."""
    stage = stage_mod
    big = small(70, 300, 150_000, 8, R=350_000, iters=40, tenure=5)
    smalls = [small(71 + s, 20 + 3 * s, 500 + 211 * s, 3 + s % 5, iters=25) for s in range(24)]
    insts = [big] + smalls
    with stage.Context(device=0, profile=True) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
        reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
        first = ctx.tabu_batch(reqs)
        assert ctx.kernel_stats("batch_gang_max")[0] > 1
        again = ctx.tabu_batch(reqs)
        for a, b in zip(first, again):
            same(a, b)
        for rq, g in zip(reqs, first):
            same(g, ctx.tabu_run(rq["inst"], rq["K"], rq["R"], rq["iters"], rq["tenure"]))
    cost = oracle.cost_table(big.base_xy, big.pick_xy, big.drop_xy, 16)
    same(first[0], oracle.tabu(cost, big.K, big.R, big.iters, big.tenure, nthreads=16))


def test_searches_the_launch_does_not_take(stage_mod):
    """More than 2048 bases, or K above 256: those searches run alone after
    the launch, the others inside it; all equal their solo runs."""
    stage = stage_mod
    wide = small(60, 2100, 700, 6, iters=8)        # 2100 bases: longer rows than the body takes
    many = small(61, 400, 3000, 300, iters=6)      # K = 300 open bases
    mid = small(62, 60, 9000, 7, iters=20)
    with stage.Context(device=0, profile=True) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in (wide, many, mid)]
        reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, (wide, many, mid))]
        got = ctx.tabu_batch(reqs)
        assert ctx.kernel_stats("batch_searches")[0] == 1
        for rq, g in zip(reqs, got):
            same(g, ctx.tabu_run(rq["inst"], rq["K"], rq["R"], rq["iters"], rq["tenure"]))
    cost = oracle.cost_table(mid.base_xy, mid.pick_xy, mid.drop_xy, 8)
    same(got[2], oracle.tabu(cost, mid.K, mid.R, mid.iters, mid.tenure, nthreads=8))


def test_malformed_batches_are_refused(stage_mod):
    stage = stage_mod
    a, b = small(80, 30, 2000, 4), small(81, 25, 1000, 3)
    with stage.Context(device=0) as ctx:
        ha, hb = (ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in (a, b))
        ok = dict(inst=ha, K=4, R=a.R, iters=5, tenure=2)
        with pytest.raises(stage.StageError) as e:
            ctx.tabu_batch([ok, dict(ok)])                      # one instance twice
        assert e.value.status == -1
        with pytest.raises(stage.StageError) as e:
            ctx.tabu_batch([ok, dict(inst=hb + 1000, K=3, R=b.R, iters=5, tenure=2)])
        assert e.value.status == -8                             # unknown instance
        with pytest.raises(stage.StageError) as e:
            ctx.tabu_batch([ok, dict(inst=hb, K=0, R=b.R, iters=5, tenure=2)])
        assert e.value.status == -1
        assert ctx.tabu_batch([]) == []
        # the context still searches correctly
        same(ctx.tabu_batch([ok])[0], ctx.tabu_run(ha, 4, a.R, 5, 2))


def test_one_poll_limit_gives_up_or_is_exact(stage_mod):
    """The waits between a search's CTAs are bounded: under a one-poll limit
    the call either reports STAGE_ERR_TIMEOUT or returns the exact results,
    and a context with the default limit then searches exactly."""
    stage = stage_mod
    big = small(90, 200, 90_000, 6, iters=20)
    insts = [big] + [small(91 + s, 40, 3000, 5, iters=15) for s in range(6)]
    wants = [oracle.tabu(oracle.cost_table(i.base_xy, i.pick_xy, i.drop_xy, 16), i.K, i.R, i.iters, i.tenure,
                         nthreads=16) for i in insts]
    outcomes = []
    with stage.Context(device=0, spin_limit=1) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
        reqs = [dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure) for h, i in zip(hs, insts)]
        for _ in range(3):
            try:
                got = ctx.tabu_batch(reqs)
                for g, w in zip(got, wants):
                    same(g, w)
                outcomes.append("ok")
            except stage.StageError as e:
                assert e.status == -5, e
                outcomes.append("timeout")
    assert len(outcomes) == 3
    with stage.Context(device=0) as ctx:
        hs = [ctx.load_instance(i.base_xy, i.pick_xy, i.drop_xy) for i in insts]
        got = ctx.tabu_batch([dict(inst=h, K=i.K, R=i.R, iters=i.iters, tenure=i.tenure)
                              for h, i in zip(hs, insts)])
    for g, w in zip(got, wants):
        same(g, w)
