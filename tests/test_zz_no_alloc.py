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
