"""Heterogeneous fleet (rotary- and fixed-wing vehicles, helipads, rotary-only
missions) on the GPU against the oracle: whole trajectories, best and final
placements per vehicle type, integers with zero tolerance.  Includes the
reductions to the identical-vehicle search and the paper's own fleet on
Eq. 1 legs.
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


def small(seed, B, M, K, R=700_000):
    lay = synth.Layout(600_000, 500_000, clustered=True, sigma_m=40_000.0)
    return synth.make_instance(f"f{seed}", seed, B, 2 * B, M, K, R, 30, 3, lay)


def check(ctx, inst, cost, heli, rot, Kr, Kf, iters, tenure, haversine=False, **kw):
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, haversine=haversine)
    got = ctx.fleet_tabu(h, Kr, Kf, inst.R, iters, tenure, heli, rot, **kw)
    ctx.unload_instance(h)
    okw = {k: v for k, v in kw.items() if k in ("start_rotary", "start_fixed", "accept_worsening")}
    want = oracle.fleet_tabu(cost, heli, rot, Kr, Kf, inst.R, iters, tenure, eval_mode="table", nthreads=8, **okw)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
    assert (got.best_cov, got.best_dist, got.best_iter) == (want.best_cov, want.best_dist, want.best_iter)
    assert np.array_equal(got.best_rotary, want.best_rotary) and np.array_equal(got.best_fixed, want.best_fixed)
    assert np.array_equal(got.final_rotary, want.final_rotary) and np.array_equal(got.final_fixed, want.final_fixed)
    assert (got.final_cov, got.final_dist) == (want.final_cov, want.final_dist)
    return got


def test_reductions_to_identical_vehicles(ctx):
    inst = small(1, 40, 3000, 6)
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    heli, rot = synth.fleet_types(1, inst.B, inst.M, 10, 0.3)
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
    plain = ctx.tabu_run(h, 6, inst.R, 40, 4)
    allrot = ctx.fleet_tabu(h, 6, 0, inst.R, 40, 4, heli, rot)
    none = ctx.fleet_tabu(h, 3, 3, inst.R, 40, 4, np.zeros(inst.B, np.uint8), np.zeros(inst.M, np.uint8))
    ctx.unload_instance(h)
    assert [tuple(m) for m in allrot.moves] == [tuple(m) for m in plain.moves]
    assert [tuple(m) for m in none.moves] == [tuple(m) for m in plain.moves]
    check(ctx, inst, cost, heli, rot, 6, 0, 40, 4)


@pytest.mark.parametrize("B,M,Kr,Kf,nh,frac,seed", [(30, 2000, 3, 2, 8, 0.3, 2), (50, 9000, 5, 3, 15, 0.2, 3),
                                                    (25, 300, 2, 4, 6, 0.5, 4), (60, 17000, 8, 4, 20, 0.3, 5),
                                                    (20, 800, 1, 1, 5, 0.9, 6)])
def test_random_fleets(ctx, B, M, Kr, Kf, nh, frac, seed):
    inst = small(10 + seed, B, M, Kr + Kf)
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    heli, rot = synth.fleet_types(seed, B, M, nh, frac)
    check(ctx, inst, cost, heli, rot, Kr, Kf, 40, 4)


def test_edges_start_and_improving_only(ctx):
    inst = small(30, 35, 4000, 5)
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    heli, rot = synth.fleet_types(7, inst.B, inst.M, 9, 0.3)
    check(ctx, inst, cost, heli, rot, 0, 4, 25, 3)                       # no rotary-wing vehicle
    check(ctx, inst, cost, heli, np.zeros(inst.M, np.uint8), 2, 3, 25, 3)  # no rotary-only mission
    check(ctx, inst, cost, heli, rot, 3, 2, 60, 2, accept_worsening=False)
    aer = [b for b in range(inst.B) if not heli[b]]
    start_r, start_f = [int(np.flatnonzero(heli)[0]), aer[0]], aer[1:4]
    check(ctx, inst, cost, heli, rot, 2, 3, 25, 3, start_rotary=start_r, start_fixed=start_f)


def test_bad_fixed_start(ctx):
    from paper_2001_05291_gb300 import stage
    inst = small(31, 20, 500, 3)
    heli, rot = synth.fleet_types(8, inst.B, inst.M, 5, 0.3)
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
    hb = int(np.flatnonzero(heli)[0])
    aer = [b for b in range(inst.B) if not heli[b]]
    with pytest.raises(stage.StageError) as e:
        ctx.fleet_tabu(h, 1, 2, inst.R, 5, 2, heli, rot, start_rotary=[aer[0]], start_fixed=[aer[1], hb])
    assert e.value.status == -1
    ctx.unload_instance(h)


def test_paper_fleet_on_eq1_legs(ctx):
    inst, heli, rot, Kr, Kf = synth.fleet_paper()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8, haversine=True)
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, haversine=True)
    assert np.array_equal(ctx.read_table(h, 0, inst.B, 0, inst.M), cost)
    ctx.unload_instance(h)
    got = check(ctx, inst, cost, heli, rot, Kr, Kf, 100, 7, haversine=True)
    assert not any(heli[b] for b in got.final_fixed)


@pytest.fixture(scope="module")
def ictx():
    """Both searches of the fleet keep their swap terms across moves (the
    incremental neighbourhood: one full pass each, then the records of the
    missions each move touched; B, held after a fixed-wing move, skips its
    refresh and update)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage
    build.build()
    with stage.Context(device=0, incremental=True, profile=True) as c:
        yield c


@pytest.mark.parametrize("B,M,Kr,Kf,nh,frac,seed", [(30, 2000, 3, 2, 8, 0.3, 2), (50, 9000, 5, 3, 15, 0.2, 3),
                                                    (60, 17000, 8, 4, 20, 0.3, 5), (20, 800, 1, 1, 5, 0.9, 6)])
def test_incremental_fleets(ictx, B, M, Kr, Kf, nh, frac, seed):
    inst = small(10 + seed, B, M, Kr + Kf)
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    heli, rot = synth.fleet_types(seed, B, M, nh, frac)
    check(ictx, inst, cost, heli, rot, Kr, Kf, 60, 4)


def test_incremental_fleet_edges(ictx):
    inst = small(30, 35, 4000, 5)
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 8)
    heli, rot = synth.fleet_types(7, inst.B, inst.M, 9, 0.3)
    check(ictx, inst, cost, heli, rot, 0, 4, 25, 3)                       # no rotary-wing vehicle
    check(ictx, inst, cost, heli, np.zeros(inst.M, np.uint8), 2, 3, 25, 3)  # no rotary-only mission
    check(ictx, inst, cost, heli, rot, 3, 2, 60, 2, accept_worsening=False)
    check(ictx, inst, cost, heli, rot, 5, 0, 30, 3)                       # rotary-wing only
    assert ictx.kernel_stats("swap_delta")[0] > 0
