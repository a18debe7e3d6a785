"""GPU path (through the C ABI) against the CPU oracle, element by element.

All quantities are integers: the bar is bit-exact equality.  Sizes span several
swap-evaluation tiles (16,384 missions per block, 8 candidate rows per block)
with ragged tails, plus the edge cases of the method: K = 1, K = B - 1, no
candidate base, unavailable bases, tiny M, M not a multiple of 4, the largest K.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05291_gb300 import synth

pytestmark = pytest.mark.gpu

INF = 2**31 - 1


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage
    build.build()
    c = stage.Context(device=0, profile=True)
    yield c
    c.close()


def load(ctx, inst, avail=None):
    return ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, avail)


def small(seed, B, M, K, R=None, clustered=True):
    lay = synth.Layout(400_000, 300_000, clustered=clustered, sigma_m=25_000.0)
    R = R if R is not None else 350_000
    return synth.make_instance(f"s{seed}", seed, B, 2 * B, M, K, R, 40, 4, lay)


def oracle_table(inst, threads=8):
    return oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, threads)


# ---------------------------------------------------------------- cost table
@pytest.mark.parametrize("name", ["tiny", "province"])
def test_cost_table_full(ctx, name):
    inst = synth.by_name(name)
    h = load(ctx, inst)
    M_pad = (inst.M + 63) // 64 * 64
    got = ctx.read_table(h, 0, inst.B, 0, M_pad)
    want = oracle_table(inst)
    assert np.array_equal(got[:, : inst.M], want)
    assert np.all(got[:, inst.M:] == INF)
    ctx.unload_instance(h)


@pytest.mark.parametrize("M", [1, 3, 63, 64, 65, 1000, 16385])
def test_cost_table_ragged(ctx, M):
    inst = small(11, 9, M, 3)
    h = load(ctx, inst)
    got = ctx.read_table(h, 0, inst.B, 0, M)
    assert np.array_equal(got, oracle_table(inst))
    ctx.unload_instance(h)


def test_cost_table_extreme_coordinates(ctx):
    lim = 2**24
    base = np.array([[-lim, -lim], [lim, lim], [0, 0], [lim, -lim]], dtype=np.int32)
    pick = np.array([[lim, lim], [-lim, lim], [3, 4], [-lim, -lim], [12345, -9876]], dtype=np.int32)
    drop = np.array([[-lim, -lim], [lim, -lim], [6, 8], [lim, lim], [-lim, 0]], dtype=np.int32)
    h = ctx.load_instance(base, pick, drop)
    got = ctx.read_table(h, 0, 4, 0, 5)
    assert np.array_equal(got, oracle.cost_table(base, pick, drop))
    ctx.unload_instance(h)


# ---------------------------------------------------------------- ranking / evaluation
@pytest.mark.parametrize("name", ["tiny", "province"])
def test_rank_and_evaluate(ctx, name):
    inst = synth.by_name(name)
    h = load(ctx, inst)
    cost = oracle_table(inst)
    for K in (1, inst.K, inst.B - 1):
        got, rs = ctx.rank_bases(h, K, inst.B)
        want, wrs = oracle.rank(cost, K)
        assert np.array_equal(got, want) and np.array_equal(rs, wrs)
    o = want[: inst.K]
    for R in (0, inst.R // 2, inst.R, INF - 1):
        assert ctx.evaluate_placement(h, o, R) == oracle.evaluate(cost, o, R)
    ctx.unload_instance(h)


def test_rank_with_unavailable_and_ties(ctx):
    inst = small(21, 30, 500, 5)
    # duplicate bases produce equal row sums: ties go to the lower index
    base = np.concatenate([inst.base_xy, inst.base_xy[[3, 7, 7]]], axis=0)
    avail = np.ones(base.shape[0], dtype=np.uint8)
    avail[[0, 5, 31]] = 0
    h = ctx.load_instance(base, inst.pick_xy, inst.drop_xy, avail)
    cost = oracle.cost_table(base, inst.pick_xy, inst.drop_xy)
    for K in (1, 4, 12, int(avail.sum())):
        got, rs = ctx.rank_bases(h, K, base.shape[0])
        want, wrs = oracle.rank(cost, K, avail)
        assert np.array_equal(got, want) and np.array_equal(rs, wrs)
    ctx.unload_instance(h)


# ---------------------------------------------------------------- swap neighbourhood
def check_swaps(ctx, h, cost, open_, R, avail=None):
    B = cost.shape[0]
    gc, gd = ctx.evaluate_swaps(h, open_, R, B)
    wc, wd = oracle.swap_table(cost, open_, R, avail, nthreads=8)
    for k, i in enumerate(open_):
        assert np.array_equal(gc[k], wc[i]), f"covered, slot {k}"
        assert np.array_equal(gd[k], wd[i]), f"distance, slot {k}"


@pytest.mark.parametrize("B,M,K", [(20, 200, 5), (37, 16384 + 20, 7), (12, 33000, 1), (9, 5000, 8),
                                   (60, 40000, 17)])
def test_swap_neighbourhood(ctx, B, M, K):
    inst = small(B * 7 + M, B, M, K)
    h = load(ctx, inst)
    cost = oracle_table(inst)
    open_, _ = oracle.rank(cost, K)
    for R in (inst.R, 150_000, INF - 1):
        check_swaps(ctx, h, cost, open_, R)
    ctx.unload_instance(h)


def test_swap_large_costs_near_range(ctx):
    """Costs spread up to about 2.5e7 m with R around 2^24, so that many terms
    near R (the largest values the per-block sums carry) occur: the
    neighbourhood table and a Tabu trajectory equal the oracle."""
    rng = np.random.default_rng(2024)
    B, M, K = 40, 6000, 6
    base = rng.integers(0, 6_000_000, size=(B, 2), dtype=np.int64).astype(np.int32)
    pick = rng.integers(0, 6_000_000, size=(M, 2), dtype=np.int64).astype(np.int32)
    drop = rng.integers(0, 6_000_000, size=(M, 2), dtype=np.int64).astype(np.int32)
    h = ctx.load_instance(base, pick, drop)
    cost = oracle.cost_table(base, pick, drop, 8)
    open_, _ = oracle.rank(cost, K)
    for R in ((1 << 24) - 3, (1 << 24) - 2, (1 << 24) - 1, 1 << 24):
        assert ((cost >= R - 2_000_000) & (cost <= R)).any()
        check_swaps(ctx, h, cost, open_, R)
    for R in ((1 << 24) - 2, (1 << 24) - 1):
        check_tabu(ctx, h, cost, K, R, 25, 4)
    ctx.unload_instance(h)


def test_swap_neighbourhood_unavailable(ctx):
    inst = small(5, 25, 3000, 6)
    avail = np.ones(inst.B, dtype=np.uint8)
    avail[[1, 2, 20]] = 0
    h = load(ctx, inst, avail)
    cost = oracle_table(inst)
    open_, _ = oracle.rank(cost, 6, avail)
    check_swaps(ctx, h, cost, open_, inst.R, avail)
    ctx.unload_instance(h)


def test_swap_neighbourhood_province(ctx):
    inst = synth.province()
    h = load(ctx, inst)
    cost = oracle_table(inst)
    open_, _ = oracle.rank(cost, inst.K)
    check_swaps(ctx, h, cost, open_, inst.R)
    ctx.unload_instance(h)


# ---------------------------------------------------------------- incremental refresh
def test_refresh_equals_full_recompute(ctx):
    inst = small(77, 40, 9000, 6)
    h = load(ctx, inst)
    cost = oracle_table(inst)
    start, _ = oracle.rank(cost, 6)
    ref = oracle.tabu(cost, 6, inst.R, 30, 3, start_open=start)
    O = list(start)
    for steps in range(0, 31, 3):
        if steps:
            for (_, i, j, *_r) in ref.moves[steps - 3: steps]:
                O = [j if x == i else x for x in O]
        a, b, b1, b2 = ctx.best_two(h, start, inst.R, inst.M, tabu_steps=steps, tenure=3)
        wa, wb, wb1, wb2 = oracle.best_two(cost, O)
        assert np.array_equal(a, wa) and np.array_equal(b, wb)
        assert np.array_equal(b1, wb1) and np.array_equal(b2, wb2)
    ctx.unload_instance(h)


# ---------------------------------------------------------------- Tabu trajectories
def check_tabu(ctx, h, cost, K, R, iters, tenure, avail=None, **kw):
    got = ctx.tabu_run(h, K, R, iters, tenure, **kw)
    okw = {k: v for k, v in kw.items() if k in ("start_open", "accept_worsening")}
    want = oracle.tabu(cost, K, R, iters, tenure, avail=avail, nthreads=8, **okw)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    assert got.n_moves == len(want.moves)
    assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist, want.best_iter)
    assert np.array_equal(got.best_open, want.best_open)
    assert np.array_equal(got.final_open, want.final_open)
    assert (got.final_cov, got.final_dist) == (want.final_cov, want.final_dist)
    return got


def test_tabu_tiny_workload(ctx):
    inst = synth.tiny()
    h = load(ctx, inst)
    cost = oracle_table(inst)
    got = check_tabu(ctx, h, cost, inst.K, inst.R, inst.iters, inst.tenure)
    _, oc, od, _ = oracle.bruteforce(cost, inst.K, inst.R)
    assert (got.best_cov, got.best_dist) == (oc, od)
    ctx.unload_instance(h)


def test_tabu_province_workload(ctx):
    inst = synth.province()
    h = load(ctx, inst)
    check_tabu(ctx, h, oracle_table(inst), inst.K, inst.R, inst.iters, inst.tenure)
    ctx.unload_instance(h)


@pytest.mark.parametrize("B,M,K,tenure,aw", [
    (20, 200, 1, 2, True), (15, 777, 14, 3, True), (30, 20000, 5, 0, True), (30, 2051, 5, 6, False),
    (48, 17000, 9, 4, True), (8, 3, 3, 2, True)])
def test_tabu_edge_cases(ctx, B, M, K, tenure, aw):
    inst = small(B + 1000 * K + M, B, M, K)
    h = load(ctx, inst)
    check_tabu(ctx, h, oracle_table(inst), K, inst.R, 60, tenure, accept_worsening=aw)
    ctx.unload_instance(h)


def test_tabu_no_candidates(ctx):
    inst = small(3, 4, 100, 4)
    h = load(ctx, inst)
    got = ctx.tabu_run(h, 4, inst.R, 10, 2)
    assert got.n_moves == 0 and got.moves == []
    assert (got.best_cov, got.best_dist) == oracle.evaluate(oracle_table(inst), np.arange(4), inst.R)
    ctx.unload_instance(h)


def test_tabu_unavailable_and_start(ctx):
    inst = small(9, 35, 6000, 6)
    avail = np.ones(inst.B, dtype=np.uint8)
    avail[[0, 4, 9, 30]] = 0
    h = load(ctx, inst, avail)
    cost = oracle_table(inst)
    start = np.array([1, 2, 3, 5, 6, 7], dtype=np.int32)
    check_tabu(ctx, h, cost, 6, inst.R, 50, 3, avail=avail, start_open=start)
    check_tabu(ctx, h, cost, 6, inst.R, 50, 3, avail=avail)
    ctx.unload_instance(h)


def test_tabu_max_K(ctx):
    inst = small(4, 1100, 700, 1024, R=200_000)
    h = load(ctx, inst)
    check_tabu(ctx, h, oracle_table(inst), 1024, inst.R, 8, 2)
    ctx.unload_instance(h)


def test_tabu_resume_equals_uninterrupted(ctx):
    inst = small(31, 40, 8000, 7)
    h = load(ctx, inst)
    full = ctx.tabu_run(h, 7, inst.R, 40, 5)
    first = ctx.tabu_run(h, 7, inst.R, 17, 5, end_state=True, B=inst.B)
    second = ctx.tabu_run(h, 7, inst.R, 23, 5, resume=first.end_state)
    assert first.moves + second.moves == full.moves
    assert (second.best_cov, second.best_dist, second.best_iter) == (full.best_cov, full.best_dist, full.best_iter)
    assert np.array_equal(second.best_open, full.best_open)
    ctx.unload_instance(h)


def test_errors_are_reported(ctx):
    from paper_2001_05291_gb300 import stage
    inst = small(1, 10, 50, 3)
    h = load(ctx, inst)
    with pytest.raises(stage.StageError) as e:
        ctx.evaluate_placement(h, [1, 1, 2], inst.R)
    assert e.value.status == -1 and "twice" in e.value.message
    with pytest.raises(stage.StageError) as e:
        ctx.tabu_run(h, 11, inst.R, 5, 1)
    assert e.value.status == -1
    with pytest.raises(stage.StageError) as e:
        ctx.tabu_run(h, 3, INF, 5, 1)
    assert e.value.status == -2
    with pytest.raises(stage.StageError) as e:
        ctx.load_instance(np.array([[2**24 + 1, 0]]), inst.pick_xy, inst.drop_xy)
    assert e.value.status == -2
    ctx.unload_instance(h)
    with pytest.raises(stage.StageError) as e:
        ctx.rank_bases(h, 3)
    assert e.value.status == -8


def test_device_resident_inputs(ctx):
    import torch
    inst = synth.tiny()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (inst.base_xy, inst.pick_xy, inst.drop_xy)]
    h = ctx.load_instance(*dev)
    got = ctx.read_table(h, 0, inst.B, 0, inst.M)
    assert np.array_equal(got, oracle_table(inst))
    ctx.unload_instance(h)


def test_autotune_changes_no_result(ctx):
    from paper_2001_05291_gb300 import stage
    inst = small(41, 90, 30000, 9)
    h = load(ctx, inst)
    before = ctx.tabu_run(h, inst.K, inst.R, 25, 3)
    seg = ctx.autotune(h, inst.K, inst.R)
    assert seg in (1024, 2048, 4096, 8192, 16384)
    after = ctx.tabu_run(h, inst.K, inst.R, 25, 3)
    assert before.moves == after.moves
    ctx.unload_instance(h)
    with stage.Context(device=0, autotune=True) as c2:
        h2 = load(c2, inst)
        tuned = c2.tabu_run(h2, inst.K, inst.R, 25, 3)
        assert tuned.moves == before.moves
    want = oracle.tabu(oracle_table(inst), inst.K, inst.R, 25, 3, nthreads=8)
    assert [tuple(m) for m in before.moves] == [tuple(m) for m in want.moves]


def test_leg_special_values(ctx):
    """Exact squares, squares +- 1 and the range extremes, through the table build:
    each leg must be the exact integer ceiling square root (as the oracle's
    float64 ceil(sqrt) is in this range)."""
    import math
    offs = []
    for (p, q) in [(3, 4), (5, 12), (20, 21), (119, 120)]:
        for k in (1, 1000, 99991):
            offs.append((p * k, q * k))
    for s in (1, 2, 7, 4096, 2**20 + 3, 2**24, 2**25 - 1):
        offs.append((s, 1))                       # s^2 + 1
    for k in (1, 3, 100, 2000, 2895):
        offs.append((2 * k * k, 2 * k))            # (2k^2 + 1)^2 - 1
    lim = 2**24
    # base at the origin; pickup at the offset (clipped into range); drop-off at the base
    pick = np.array([(max(-lim, min(lim, dx)), max(-lim, min(lim, dy))) for dx, dy in offs], dtype=np.int32)
    base = np.array([[0, 0], [-lim, -lim]], dtype=np.int32)
    drop = np.zeros_like(pick)
    h = ctx.load_instance(base, pick, drop)
    got = ctx.read_table(h, 0, 2, 0, len(offs))
    for m, (x, y) in enumerate(pick.tolist()):
        n0 = x * x + y * y
        c0 = math.isqrt(n0) + (math.isqrt(n0) ** 2 != n0)
        n1 = (x + lim) ** 2 + (y + lim) ** 2
        c1 = math.isqrt(n1) + (math.isqrt(n1) ** 2 != n1)
        pd = c0                                    # pickup -> drop-off (drop at origin)
        assert got[0, m] == c0 + pd + 0
        dn = lim * lim * 2
        c2 = math.isqrt(dn) + (math.isqrt(dn) ** 2 != dn)
        assert got[1, m] == c1 + pd + c2
    ctx.unload_instance(h)


def test_graph_replay_and_small_block_paths():
    """Without profiling, single searches replay 16-iteration CUDA graphs (large
    instances) or run in one resident block (small ones); both equal the oracle,
    also for an iteration count that is not a multiple of 16 and for the
    improving-only rule that stops early."""
    from paper_2001_05291_gb300 import stage
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with stage.Context(device=0) as c2:
        for inst, iters, aw in ((small(61, 70, 12000, 8), 45, True), (small(62, 70, 12000, 8), 200, False),
                                (synth.tiny(), 37, True), (small(63, 12, 900, 3), 50, False)):
            h = load(c2, inst)
            got = c2.tabu_run(h, inst.K, inst.R, iters, inst.tenure, accept_worsening=aw)
            want = oracle.tabu(oracle_table(inst), inst.K, inst.R, iters, inst.tenure, accept_worsening=aw,
                               nthreads=8)
            assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
            assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist, want.best_iter)
            c2.unload_instance(h)


def test_incremental_equals_full_pass():
    """STAGE_INCREMENTAL (the default for tables well beyond L2) keeps the
    neighbourhood's gain and extra terms across iterations and updates them from
    the missions whose best / second best changed, and rebuilds the closed
    base's column in the refresh; STAGE_FULL_PASS re-evaluates the whole table every iteration.  The
    persistent launch (the default), the per-kernel launches of the incremental
    form (STAGE_NO_PERSIST) and the full pass all equal the oracle's trajectory: several K (1 to 64), unavailable bases, a
    start placement, the improving-only rule, R below most costs and R near
    INT32_MAX."""
    from paper_2001_05291_gb300 import stage
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [(small(71, 70, 12000, 8), 120, True, None, None),
             (small(72, 110, 24000, 17, R=150_000), 50, True, None, None),
             (small(73, 45, 20000, 1), 40, True, None, None),
             (small(74, 60, 9000, 5), 80, False, [3, 7, 20, 41], None),
             (small(75, 50, 8000, 6, R=2**31 - 2), 30, True, None, None),
             (small(76, 300, 5000, 64), 25, True, None, np.arange(64, dtype=np.int32) * 4)]
    with stage.Context(device=0, incremental=True) as ci, stage.Context(device=0, profile=True, incremental=True) as cp, \
            stage.Context(device=0, full_pass=True) as cf, \
            stage.Context(device=0, profile=True, incremental=True, persist=False) as cn:
        for inst, iters, aw, unavail, start in cases:
            avail = None
            if unavail is not None:
                avail = np.ones(inst.B, dtype=np.uint8)
                avail[unavail] = 0
            cost = oracle_table(inst)
            okw = {"start_open": start} if start is not None else {}
            want = oracle.tabu(cost, inst.K, inst.R, iters, inst.tenure, avail=avail, accept_worsening=aw,
                               nthreads=8, **okw)
            for c in (ci, cp, cf, cn):
                h = load(c, inst, avail)
                got = c.tabu_run(h, inst.K, inst.R, iters, inst.tenure, accept_worsening=aw, **okw)
                assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
                assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist,
                                                                        want.best_iter)
                assert (got.final_cov, got.final_dist) == (want.final_cov, want.final_dist)
                c.unload_instance(h)
        # the persistent launch by default, the per-iteration launches with
        # STAGE_NO_PERSIST, no incremental update with STAGE_FULL_PASS
        assert cp.kernel_stats("persist")[0] == len(cases) and cp.kernel_stats("swap_delta")[0] == 0
        assert cn.kernel_stats("swap_delta")[0] > 0 and cn.kernel_stats("persist")[0] == 0
        assert cf.kernel_stats("swap_delta")[0] == 0 and cf.kernel_stats("persist")[0] == 0


def test_incremental_edge_cases_and_resume():
    """The incremental form on the edge cases of the Tabu tests (K = 1, K = B - 1,
    tenure 0, improving-only, M = 3) and across a resume (an odd start
    iteration), on its per-kernel path and its persistent launch."""
    from paper_2001_05291_gb300 import stage
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with stage.Context(device=0, profile=True, incremental=True, persist=False) as cp, \
            stage.Context(device=0, incremental=True) as cg:
        for B, M, K, tenure, aw in [(20, 200, 1, 2, True), (15, 777, 14, 3, True), (30, 20000, 5, 0, True),
                                    (30, 2051, 5, 6, False), (48, 17000, 9, 4, True), (8, 3, 3, 2, True)]:
            inst = small(B + 1000 * K + M, B, M, K)
            cost = oracle_table(inst)
            for c in (cp, cg):
                h = load(c, inst)
                check_tabu(c, h, cost, K, inst.R, 60, tenure, accept_worsening=aw)
                c.unload_instance(h)
        inst = small(31, 40, 8000, 7)
        for c in (cp, cg):
            h = load(c, inst)
            full = c.tabu_run(h, 7, inst.R, 40, 5)
            first = c.tabu_run(h, 7, inst.R, 17, 5, end_state=True, B=inst.B)
            second = c.tabu_run(h, 7, inst.R, 23, 5, resume=first.end_state)
            assert [tuple(m) for m in first.moves + second.moves] == [tuple(m) for m in full.moves]
            assert (second.best_cov, second.best_dist, second.best_iter) == (full.best_cov, full.best_dist,
                                                                             full.best_iter)
            c.unload_instance(h)
