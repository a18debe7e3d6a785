"""The one-pass table build (table, row sums, mission-major copy and its cell
minima together), taken by a context whose searches use the incremental
neighbourhood, against the CPU oracle.

Integers throughout: tables and row sums are compared exactly (Haversine legs
within one metre, as in the geo tests).  Sizes cover base counts that are not a
multiple of the 32-position cells or of the 8-cell blocks, mission counts with
ragged tails, the coordinate extremes, and a ranking after an instance update
(whose row sums the update makes stale).  The copy and its minima are checked
through the searches that read them: the incremental trajectories equal the
oracle's.
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
    return synth.make_instance(f"f{seed}", seed, B, 2 * B, M, K, R, 25, 4, lay)


@pytest.mark.parametrize("B,M", [(1, 1), (37, 65), (300, 20_000), (257, 4_097), (1000, 3_000)])
def test_fused_table_and_rank(stage_mod, B, M):
    inst = small(B + M, B, M, min(5, B))
    want = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    with stage_mod.Context(device=0, incremental=True, profile=True) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        assert ctx.kernel_stats("transpose")[0] == 0   # no separate copy pass
        got = ctx.read_table(h, 0, B, 0, M)
        assert np.array_equal(got, want)
        for K in sorted({1, min(5, B), B}):
            open_, rs = ctx.rank_bases(h, K, B)
            wo, wrs = oracle.rank(want, K)
            assert np.array_equal(open_, wo) and np.array_equal(rs, wrs)
        assert ctx.kernel_stats("rowsum")[0] == 0      # the sums came with the table
        ctx.unload_instance(h)


def test_fused_table_extreme_coordinates(stage_mod):
    lim = 2**24
    base = np.array([[-lim, -lim], [lim, lim], [0, 0], [lim, -lim], [-lim, lim]], dtype=np.int32)
    pick = np.array([[lim, lim], [-lim, lim], [3, 4], [-lim, -lim], [12345, -9876]], dtype=np.int32)
    drop = np.array([[-lim, -lim], [lim, -lim], [6, 8], [lim, lim], [-lim, 0]], dtype=np.int32)
    with stage_mod.Context(device=0, incremental=True) as ctx:
        h = ctx.load_instance(base, pick, drop)
        want = oracle.cost_table(base, pick, drop)
        assert np.array_equal(ctx.read_table(h, 0, 5, 0, 5), want)
        open_, rs = ctx.rank_bases(h, 2, 5)
        wo, wrs = oracle.rank(want, 2)
        assert np.array_equal(open_, wo) and np.array_equal(rs, wrs)


def test_fused_table_haversine(stage_mod):
    inst = synth.geo_instance("gf", 4, 150, 5000, 8, 1_500_000, 10, 5)
    want = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8, haversine=True)
    with stage_mod.Context(device=0, incremental=True) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, haversine=True)
        got = ctx.read_table(h, 0, inst.B, 0, inst.M)
    diff = np.abs(got.astype(np.int64) - want.astype(np.int64))
    assert diff.max() <= 1


def test_rank_after_update_recomputes_row_sums(stage_mod):
    inst = small(77, 120, 2000, 6)
    extra = small(78, 120, 300, 6)
    with stage_mod.Context(device=0, incremental=True, profile=True) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        ctx.update_instance(h, add_pick=extra.pick_xy, add_drop=extra.drop_xy, remove=[3, 10, 999])
        pick = np.concatenate([inst.pick_xy, extra.pick_xy])
        drop = np.concatenate([inst.drop_xy, extra.drop_xy])
        keep = np.ones(len(pick), bool)
        keep[[3, 10, 999]] = False
        want = oracle.cost_table(inst.base_xy, pick[keep], drop[keep], 8)
        open_, rs = ctx.rank_bases(h, inst.K, inst.B)
        wo, wrs = oracle.rank(want, inst.K)
        assert np.array_equal(open_, wo) and np.array_equal(rs, wrs)
        assert ctx.kernel_stats("rowsum")[0] == 1
        # and the search, on the refreshed copy, follows the oracle
        got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
        wt = oracle.tabu(want, inst.K, inst.R, inst.iters, inst.tenure)
        assert [tuple(m) for m in got.moves] == [tuple(m) for m in wt.moves]


def test_fused_copy_feeds_the_persistent_search(stage_mod):
    inst = small(91, 700, 60_000, 12)
    want = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    wt = oracle.tabu(want, inst.K, inst.R, 60, inst.tenure, nthreads=8)
    with stage_mod.Context(device=0, incremental=True, profile=True) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        got = ctx.tabu_run(h, inst.K, inst.R, 60, inst.tenure)
        assert ctx.kernel_stats("transpose")[0] == 0
        assert ctx.kernel_stats("persist")[0] == 1
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in wt.moves]
