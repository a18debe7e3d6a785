"""Haversine legs (Eq. 1) on the GPU against the oracle.

The two sides evaluate the same double-precision expression in the same order
(no fused multiply-add on either side) with their own sine, cosine and arcsine;
a leg can differ only when its distance lies within a few units in the last
place of a whole metre.  The table check allows a one-metre difference and
counts them (none is expected at these sizes); the searches are compared on
instances whose two tables are identical, which the tests assert first.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05291_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage
    build.build()
    with stage.Context(device=0) as c:
        yield c


def geo_table(inst):
    return oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8, haversine=True)


def gpu_table(ctx, h, inst):
    return ctx.read_table(h, 0, inst.B, 0, inst.M)


@pytest.mark.parametrize("seed,B,M", [(1, 40, 3000), (2, 378, 180), (3, 150, 20000)])
def test_table_matches_oracle(ctx, seed, B, M):
    inst = synth.geo_instance("g", seed, B, M, 8, 1_500_000, 10, 5)
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, haversine=True)
    got = gpu_table(ctx, h, inst)
    ctx.unload_instance(h)
    want = geo_table(inst)
    diff = np.abs(got.astype(np.int64) - want.astype(np.int64))
    assert diff.max() <= 1
    assert int((diff != 0).sum()) <= max(1, got.size // 1_000_000)


def test_paper_scale_search(ctx):
    """The paper's scale (378 bases, 180 missions, 12 vehicles) on Eq. 1 legs:
    ranking, Tabu trajectory and local search equal the oracle's."""
    inst = synth.geo_paper()
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, haversine=True)
    cost = geo_table(inst)
    assert np.array_equal(gpu_table(ctx, h, inst), cost)
    start, rs = ctx.rank_bases(h, inst.K, inst.B)
    wo, wrs = oracle.rank(cost, inst.K)
    assert np.array_equal(start, wo) and np.array_equal(rs, wrs)
    got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
    want = oracle.tabu(cost, inst.K, inst.R, inst.iters, inst.tenure, nthreads=8)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist, want.best_iter)
    ps, pc = synth.scan_orders(5, 6, inst.K, inst.B - inst.K)
    ls = ctx.local_search(h, inst.K, inst.R, ps, pc)
    lw = oracle.local_search(cost, inst.K, inst.R, ps, pc)
    assert [tuple(m) for m in ls.moves] == [tuple(m) for m in lw.moves]
    ctx.unload_instance(h)


def test_batch_inline_and_appended_missions(ctx):
    inst = synth.geo_instance("g", 7, 60, 4000, 6, 1_200_000, 40, 4)
    cost = geo_table(inst)
    # an inline request in the batch engine equals the search alone and the oracle
    t = ctx.batch_submit([dict(base_xy=inst.base_xy, pick_xy=inst.pick_xy, drop_xy=inst.drop_xy, K=6,
                               R=inst.R, iters=40, tenure=4, haversine=True)])[0]
    got = t.wait()
    want = oracle.tabu(cost, 6, inst.R, 40, 4, nthreads=8)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    # appended missions take Eq. 1 legs too
    h = ctx.load_instance(inst.base_xy, inst.pick_xy[:3000], inst.drop_xy[:3000], haversine=True)
    ctx.update_instance(h, add_pick=inst.pick_xy[3000:], add_drop=inst.drop_xy[3000:])
    assert np.array_equal(ctx.read_table(h, 0, inst.B, 0, inst.M), cost)
    ctx.unload_instance(h)


def test_coordinate_ranges(ctx):
    from paper_2001_05291_gb300 import stage
    inst = synth.geo_instance("g", 9, 10, 30, 3, 1_000_000, 5, 2)
    bad = inst.pick_xy.copy()
    bad[3, 0] = 90_000_001                       # latitude beyond the pole
    with pytest.raises(stage.StageError) as e:
        ctx.load_instance(inst.base_xy, bad, inst.drop_xy, haversine=True)
    assert e.value.status == -2
    ok = inst.pick_xy.copy()
    ok[3] = (90_000_000, 180_000_000)            # the pole and the antimeridian are inside
    h = ctx.load_instance(inst.base_xy, ok, inst.drop_xy, haversine=True)
    ctx.unload_instance(h)
    with pytest.raises(stage.StageError):        # microdegree values are out of range as metres
        ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
