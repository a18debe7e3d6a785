"""The allocation-free swap evaluation (stage_evaluate_swaps_noalloc) against the
allocating one (stage_evaluate_swaps), both through the C ABI.

Some callers cannot allocate device memory: a re-staging service embedded in a
host application that owns all device memory through its own fixed pool, or a
dispatch loop that must not block on cudaMalloc or run out of memory halfway
through a request.  For them the engine has one call whose scratch is a static
device array; the caller passes inputs and outputs in device memory.  All
results are integers, so the tolerance is zero: both calls must agree exactly,
on two calls in a row (the second must not see what the first left behind).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05291_gb300 import build, stage, synth
    build.build()
    ctx = stage.Context(device=0)
    yield torch, stage, synth, ctx
    ctx.close()


def test_noalloc_matches_allocating_call_twice(setup):
    torch, stage, synth, ctx = setup
    inst = synth.province()
    B, M, K = inst.B, inst.M, inst.K
    M_pad = (M + 63) // 64 * 64
    avail = np.ones(B, dtype=np.uint8)
    avail[[3, 50, 299]] = 0
    h_all = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
    h_av = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy, avail)
    table = ctx.read_table(h_all, 0, B, 0, M_pad)          # pads hold INT32_MAX
    cost = torch.from_numpy(table).cuda()
    open1, _ = ctx.rank_bases(h_all, K)
    open2, _ = ctx.rank_bases(h_av, K)
    open2 = open2[::-1].copy()                               # another slot order
    cases = [(h_all, open1, inst.R, None), (h_av, open2, inst.R // 2, avail)]
    for h, open_, R, av in cases:
        want_c, want_d = ctx.evaluate_swaps(h, open_, R, B)
        out_c = torch.full((K, B), 7, dtype=torch.int64, device="cuda")
        out_d = torch.full((K, B), 7, dtype=torch.int64, device="cuda")
        d_open = torch.from_numpy(np.ascontiguousarray(open_, dtype=np.int32)).cuda()
        d_av = None if av is None else torch.from_numpy(av).cuda()
        stage.evaluate_swaps_noalloc(cost, M, d_open, R, out_c, out_d, d_av)
        torch.cuda.synchronize()
        assert np.array_equal(out_c.cpu().numpy(), want_c)
        assert np.array_equal(out_d.cpu().numpy(), want_d)
    ctx.unload_instance(h_all)
    ctx.unload_instance(h_av)


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    torch, stage, synth, ctx = setup
    cost = torch.full((2, 1_000_000), 2**31 - 1, dtype=torch.int32, device="cuda")
    d_open = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((1, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(stage.StageError) as e:
        stage.evaluate_swaps_noalloc(cost, 1_000_000, d_open, 1000, out, out.clone())
    assert e.value.status == -2 and "static scratch" in e.value.message


def test_noalloc_allocates_nothing(setup):
    """The property the call exists for: after a warm-up call, further calls
    leave the device's free memory unchanged (any cudaMalloc, pinned host
    allocation or pool growth would show)."""
    torch, stage, synth, ctx = setup
    inst = synth.tiny()
    M_pad = (inst.M + 63) // 64 * 64
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
    cost = torch.from_numpy(ctx.read_table(h, 0, inst.B, 0, M_pad)).cuda()
    open_, _ = ctx.rank_bases(h, inst.K)
    ctx.unload_instance(h)
    d_open = torch.from_numpy(np.ascontiguousarray(open_, dtype=np.int32)).cuda()
    out_c = torch.empty((inst.K, inst.B), dtype=torch.int64, device="cuda")
    out_d = torch.empty_like(out_c)
    stage.evaluate_swaps_noalloc(cost, inst.M, d_open, inst.R, out_c, out_d)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        stage.evaluate_swaps_noalloc(cost, inst.M, d_open, inst.R, out_c, out_d)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_bad_placements_on_the_device(setup):
    """Ids the host cannot check (device memory): out of range, repeated or
    unavailable bases leave every output entry at -1 and read nothing outside
    the table."""
    torch, stage, synth, ctx = setup
    inst = synth.tiny()
    M_pad = (inst.M + 63) // 64 * 64
    h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
    cost = torch.from_numpy(ctx.read_table(h, 0, inst.B, 0, M_pad)).cuda()
    good, _ = ctx.rank_bases(h, inst.K)
    want_c, want_d = ctx.evaluate_swaps(h, good, inst.R, inst.B)
    ctx.unload_instance(h)
    av = np.ones(inst.B, dtype=np.uint8)
    av[int(good[1])] = 0
    bad_cases = [([*good[:-1], inst.B], None), ([*good[:-1], -3], None), ([*good[:-1], int(good[0])], None),
                 (list(good), av)]
    out_c = torch.empty((inst.K, inst.B), dtype=torch.int64, device="cuda")
    out_d = torch.empty_like(out_c)
    for open_, a in bad_cases:
        d_open = torch.tensor(open_, dtype=torch.int32, device="cuda")
        d_av = None if a is None else torch.from_numpy(a).cuda()
        stage.evaluate_swaps_noalloc(cost, inst.M, d_open, inst.R, out_c, out_d, d_av)
        torch.cuda.synchronize()
        assert (out_c.cpu().numpy() == -1).all() and (out_d.cpu().numpy() == -1).all()
        # a good call right after still gives the allocating call's result
        d_good = torch.from_numpy(np.ascontiguousarray(good, dtype=np.int32)).cuda()
        stage.evaluate_swaps_noalloc(cost, inst.M, d_good, inst.R, out_c, out_d)
        torch.cuda.synchronize()
        assert np.array_equal(out_c.cpu().numpy(), want_c) and np.array_equal(out_d.cpu().numpy(), want_d)


def test_noalloc_rejects_malformed_tensors_before_any_launch(setup):
    torch, stage, synth, ctx = setup
    B, M_pad, K = 20, 256, 4
    cost = torch.full((B, M_pad), 1000, dtype=torch.int32, device="cuda")
    d_open = torch.arange(K, dtype=torch.int32, device="cuda")
    out = torch.empty((K, B), dtype=torch.int64, device="cuda")
    bad = [
        dict(cost=cost.to(torch.int64)),                                   # table not int32
        dict(cost=cost.reshape(-1)),                                       # table not 2-D
        dict(open_=d_open.to(torch.int64)),                                # placement not int32
        dict(out_cov=out.to(torch.int32).reshape(-1)[:K * B].clone()),     # outputs not int64
        dict(out_dist=out[:, :B // 2]),                                    # too few / not contiguous
        dict(base_available=torch.ones(B, dtype=torch.uint8)),             # host tensor
        dict(base_available=torch.ones(B - 1, dtype=torch.uint8, device="cuda")),   # short
        dict(base_available=torch.ones(B, dtype=torch.int32, device="cuda")),       # not uint8
        dict(open_=d_open.cpu()),                                          # host tensor
    ]
    for kw in bad:
        args = dict(cost=cost, open_=d_open, out_cov=out, out_dist=out.clone(), base_available=None)
        args.update(kw)
        with pytest.raises(ValueError):
            stage.evaluate_swaps_noalloc(args["cost"], 200, args["open_"], 1000, args["out_cov"],
                                         args["out_dist"], args["base_available"])
