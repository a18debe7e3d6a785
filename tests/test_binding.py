"""The ctypes binding's result objects without a device: a trajectory comes back
as a structured numpy view of the library's stage_move records
(TabuResult.moves_array) and as a list of (iter, i, j, flags, cov, dist)
tuples of Python ints built from it on first use (TabuResult.moves); both
carry the same values, 64-bit fields included.  An instance update is
marshalled into counts and int32 copies of the caller's arrays, and a
malformed one is refused before the library sees it."""
import ctypes as C

import numpy as np
import pytest

from paper_2001_05291_gb300 import stage


def trajectory(rows):
    t = (stage.StageMove * max(1, len(rows)))()
    for k, (it, i, j, fl, cov, dist) in enumerate(rows):
        t[k].iter, t[k].i, t[k].j, t[k].flags, t[k].cov, t[k].dist = it, i, j, fl, cov, dist
    return t


ROWS = [(0, 3, 17, 4, 12, 345), (1, 17, 2, 0, 2**40 + 7, 2**52 - 1), (2, 9, 1, 3, -5, -(2**50))]


def test_move_records_match_the_c_layout():
    assert stage._MOVE_DTYPE.itemsize == C.sizeof(stage.StageMove)
    for name, _ in stage.StageMove._fields_:
        assert stage._MOVE_DTYPE.fields[name][1] == getattr(stage.StageMove, name).offset


def test_moves_list_and_array_agree():
    t = trajectory(ROWS)
    arr = stage._moves_array(t, len(ROWS))
    r = stage.TabuResult(len(ROWS), np.zeros(2, np.int32), 1, 2, 0, np.zeros(2, np.int32), 1, 2, arr)
    assert r.moves == ROWS
    assert all(type(v) is int for m in r.moves for v in m)
    assert r.moves is r.moves                      # built once
    assert r.moves_array["cov"].tolist() == [m[4] for m in ROWS]
    assert stage._moves(t, 2) == ROWS[:2]          # the eager form gives the same tuples
    assert "n_moves=3" in repr(r)


def test_empty_and_list_trajectories():
    assert stage.TabuResult(0, None, 0, 0, -1, None, 0, 0).moves == []
    assert stage._moves_array(None, 5).shape == (0,)
    assert stage.TabuResult(0, None, 0, 0, -1, None, 0, 0, stage._moves_array(trajectory([]), 0)).moves == []
    r = stage.TabuResult(1, None, 0, 0, 0, None, 0, 0, [ROWS[0]])
    assert r.moves == [ROWS[0]] and r.moves_array is None


def _ints(ptr, n):
    return list((C.c_int32 * n).from_address(ptr)) if n else []


def test_update_marshalling():
    """An instance update reaches the library as counts and pointers to int32
    copies of the caller's arrays, kept alive with it."""
    pick = np.array([[10, 20], [30, 40], [-5, 7]], dtype=np.int64)
    drop = [[1, 2], [3, 4], [5, 6]]
    u, keep = stage._make_update(add_pick=pick, add_drop=drop, remove=[4, 9], unavailable=np.array([2]),
                                 available=[])
    assert (u.n_add, u.n_remove, u.n_unavail, u.n_avail) == (3, 2, 1, 0)
    assert _ints(u.add_pick_xy, 6) == [10, 20, 30, 40, -5, 7]
    assert _ints(u.add_drop_xy, 6) == [1, 2, 3, 4, 5, 6]
    assert _ints(u.remove_ids, 2) == [4, 9] and _ints(u.unavail_ids, 1) == [2]
    assert all(a.dtype == np.int32 and a.flags.c_contiguous for a in keep)
    u, keep = stage._make_update()
    assert (u.n_add, u.n_remove, u.n_unavail, u.n_avail) == (0, 0, 0, 0) and keep == []
    assert not u.add_pick_xy and not u.remove_ids


def test_malformed_updates_are_refused():
    for kw in (dict(add_pick=[1, 2]), dict(add_drop=[1, 2]), dict(add_pick=[1, 2, 3, 4], add_drop=[1, 2]),
               dict(add_pick=[1, 2, 3], add_drop=[4, 5, 6])):
        with pytest.raises(ValueError):
            stage._make_update(**kw)
    with pytest.raises(ValueError):
        stage._host_i32([1, 2, 3], 4)
    assert stage._host_i32(np.arange(4, dtype=np.int64), 4).dtype == np.int32
