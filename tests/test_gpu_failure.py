"""Failure detection without a GPU fault.

* A device-side wait that runs out: one bounded wait on a flag that nothing
  sets returns STAGE_ERR_TIMEOUT (no trap, no hang) and the context stays
  usable.
* The persistent search's grid barriers under a spin limit of one poll: the
  call either gives up with STAGE_ERR_TIMEOUT or (if every CTA arrived in
  time) returns the exact result; the same context then runs the search with
  the default limit and matches the oracle.
* Allocation failures injected through the allocator hook: failing the n-th
  allocation of a load + search returns STAGE_ERR_NO_MEMORY or takes a
  documented fallback with the exact result, and nothing leaks (the context's
  accounting returns to zero, every hook allocation is freed).
"""
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


def mid_instance():
    lay = synth.Layout(400_000, 300_000, clustered=True, sigma_m=25_000.0)
    return synth.make_instance("failure", 11, 60, 120, 12000, 7, 350_000, 40, 5, lay)


def test_bounded_wait_gives_up_with_timeout(stage_mod):
    stage = stage_mod
    inst = synth.tiny()
    with stage.Context(device=0, spin_limit=1000) as ctx:
        for _ in range(2):
            with pytest.raises(stage.StageError) as e:
                ctx.test_wait_timeout()
            assert e.value.status == -5 and "gave up" in e.value.message
        # the context is still usable
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
    want = oracle.tabu(oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy), inst.K, inst.R, inst.iters,
                       inst.tenure)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]


def test_persistent_search_under_a_one_poll_limit(stage_mod):
    stage = stage_mod
    inst = mid_instance()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy)
    want = oracle.tabu(cost, inst.K, inst.R, inst.iters, inst.tenure)
    outcomes = []
    with stage.Context(device=0, incremental=True, spin_limit=1) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        for _ in range(3):
            try:
                got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
                assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
                outcomes.append("ok")
            except stage.StageError as e:
                assert e.status == -5, e
                outcomes.append("timeout")
    assert outcomes
    with stage.Context(device=0, incremental=True) as ctx:
        h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
        got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
    assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]


class FailingAllocator:
    """Torch-backed allocator hook that refuses its n-th allocation."""

    def __init__(self, stage, torch, fail_at):
        self.torch, self.fail_at, self.count, self.live = torch, fail_at, 0, {}
        self.alloc_cb = stage.ALLOC_FN(self._alloc)
        self.free_cb = stage.FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        self.count += 1
        if self.count == self.fail_at:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda:0")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, nbytes, user):
        self.live.pop(ptr, None)


def test_failed_allocations_return_no_memory_without_leaks(stage_mod):
    import torch
    stage = stage_mod
    inst = mid_instance()
    cost = oracle.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy)
    want = oracle.tabu(cost, inst.K, inst.R, inst.iters, inst.tenure)
    seen_fail, n = 0, 1
    while True:
        al = FailingAllocator(stage, torch, n)
        ctx = stage.Context(device=0, incremental=True, allocator=al)
        h = None
        try:
            h = ctx.load_instance(inst.base_xy, inst.pick_xy, inst.drop_xy)
            got = ctx.tabu_run(h, inst.K, inst.R, inst.iters, inst.tenure)
            # a refused buffer of the incremental form falls back to the full
            # pass: the result is the same
            assert [tuple(m) for m in got.moves] == [tuple(m) for m in want.moves]
            ok = True
        except stage.StageError as e:
            assert e.status == -3, e   # STAGE_ERR_NO_MEMORY
            seen_fail += 1
            ok = False
        if h is not None:
            ctx.unload_instance(h)
        assert ctx.memory_used() == 0
        ctx.close()
        assert not al.live, f"{len(al.live)} allocations leaked (failing allocation {n})"
        if al.count < n:   # the n-th allocation never happened: every position was tried
            assert ok
            break
        n += 1
    assert seen_fail >= 1
