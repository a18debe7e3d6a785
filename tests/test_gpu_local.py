"""Local search (Alg. 2 as read for identical vehicles) on the GPU against the oracle.

The whole trajectory (every applied move with its objective), the final
placement, the number of passes and the local-optimum flag must be identical:
integers, zero tolerance.  The cases span single-block and graph-replayed
driver paths, the persistent search (the whole local search in one
cooperative launch) and its per-launch form, pass changes (the step that keeps
the accumulators and skips the swap pass), budgets, unavailable bases, K = 1
and an instance with no candidate base.
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


def small(seed, B, M, K, R=None):
    lay = synth.Layout(600_000, 500_000, clustered=True, sigma_m=40_000.0)
    R = R if R is not None else 700_000
    return synth.make_instance(f"l{seed}", seed, B, 2 * B, M, K, R, 30, 3, lay)


def cost_of(inst):
    return oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)


def check(ctx, inst, K, R, passes, seed, avail=None, max_moves=100000, start_open=None):
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, avail)
    cost = cost_of(inst)
    n_avail = inst.B if avail is None else int(np.asarray(avail).sum())
    ps, pc = synth.scan_orders(seed, passes, K, n_avail - K)
    got = ctx.local_search(h, K, R, ps, pc, max_moves=max_moves, start_open=start_open)
    want = oracle.local_search(cost, K, R, ps, pc, start_open=start_open, avail=avail, max_moves=max_moves,
                               nthreads=8)
    ctx.unload_instance(h)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    assert got.n_moves == len(want.moves)
    assert np.array_equal(got.final_open, want.final_open)
    assert (got.final_cov, got.final_dist) == (want.final_cov, want.final_dist)
    assert (got.passes, got.local_optimum) == (want.passes, want.local_optimum)
    return got


def test_tiny_workload(ctx):
    inst = synth.tiny()
    got = check(ctx, inst, inst.K, inst.R, 6, 0)
    assert got.local_optimum


@pytest.mark.parametrize("B,M,K,seed", [(30, 900, 4, 1), (45, 5000, 7, 2), (60, 17000, 12, 3), (25, 33, 3, 4),
                                        (80, 2500, 20, 5), (120, 12000, 9, 6)])
def test_random_instances(ctx, B, M, K, seed):
    inst = small(100 + seed, B, M, K)
    got = check(ctx, inst, K, inst.R, 8, seed)
    assert got.passes >= 2


def test_province_workload(ctx):
    inst = synth.province()
    check(ctx, inst, inst.K, inst.R, 5, 7)


def test_budget_passes_and_start(ctx):
    inst = small(200, 50, 6000, 6)
    full = check(ctx, inst, 6, inst.R, 8, 8)
    assert full.n_moves >= 3
    cut = check(ctx, inst, 6, inst.R, 8, 8, max_moves=2)
    assert cut.n_moves == 2 and not cut.local_optimum
    check(ctx, inst, 6, inst.R, 1, 8)                        # one pass only
    check(ctx, inst, 6, inst.R, 8, 8, max_moves=0)
    check(ctx, inst, 6, inst.R, 8, 9, start_open=np.arange(6) * 3)


def test_unavailable_bases_k1_and_no_candidates(ctx):
    inst = small(300, 40, 4000, 5)
    avail = np.ones(inst.B, dtype=np.uint8)
    avail[[0, 5, 17, 33]] = 0
    got = check(ctx, inst, 5, inst.R, 6, 10, avail=avail)
    assert all(m[2] not in (0, 5, 17, 33) for m in got.moves)
    check(ctx, inst, 1, inst.R, 6, 11)
    tight = small(301, 6, 500, 6)
    got = check(ctx, tight, 6, tight.R, 2, 12)
    assert got.n_moves == 0 and got.local_optimum and got.passes == 0


def test_wide_range_and_bad_permutation(ctx):
    from paper_2001_05291_gb300 import stage
    inst = small(400, 35, 3000, 5)
    check(ctx, inst, 5, 2**31 - 2, 5, 13)                    # everything covered: distance only
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
    ps, pc = synth.scan_orders(14, 2, 5, inst.B - 5)
    pc[1, 0] = pc[1, 1]
    with pytest.raises(stage.StageError):
        ctx.local_search(h, 5, inst.R, ps, pc)
    ctx.unload_instance(h)


@pytest.fixture(scope="module", params=[True, False], ids=["persistent", "per-launch"])
def ictx(request):
    """A context whose local searches keep the swap terms across moves (the
    incremental neighbourhood: one full pass, then the records of the
    missions each move touched; a pass change holds the terms): the whole
    search in one cooperative launch, or per-step launches."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage
    build.build()
    with stage.Context(device=0, incremental=True, persist=request.param, profile=True) as c:
        c.persistent = request.param
        yield c


@pytest.mark.parametrize("B,M,K,seed", [(30, 900, 4, 1), (60, 17000, 12, 3), (80, 2500, 20, 5), (120, 12000, 9, 6)])
def test_incremental_local_search(ictx, B, M, K, seed):
    inst = small(100 + seed, B, M, K)
    got = check(ictx, inst, K, inst.R, 8, seed)
    assert got.passes >= 2


def test_incremental_local_search_edges(ictx):
    inst = small(300, 40, 4000, 5)
    avail = np.ones(inst.B, dtype=np.uint8)
    avail[[0, 5, 17, 33]] = 0
    check(ictx, inst, 5, inst.R, 6, 10, avail=avail)
    check(ictx, inst, 1, inst.R, 6, 11)
    full = small(200, 50, 6000, 6)
    cut = check(ictx, full, 6, full.R, 8, 8, max_moves=2)
    assert cut.n_moves == 2 and not cut.local_optimum
    check(ictx, full, 6, full.R, 8, 9, start_open=np.arange(6) * 3)
    check(ictx, full, 6, 2**31 - 2, 5, 13)
    if ictx.persistent:
        assert ictx.kernel_stats("local_persist")[0] > 0
    else:
        assert ictx.kernel_stats("swap_delta")[0] > 0
