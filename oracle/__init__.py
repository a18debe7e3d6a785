"""Python access to the CPU oracle (oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
package.  ``build()`` compiles oracle.c with gcc (no fast-math: the leg distance
needs the correctly rounded float64 sqrt).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

INF = 2**31 - 1
MOVE_FALLBACK, MOVE_ASPIRATION, MOVE_NEW_BEST = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (skipped when up to date)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Move(C.Structure):
    _fields_ = [("iter", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("flags", C.c_int32),
                ("cov", C.c_int64), ("dist", C.c_int64)]


class TabuIO(C.Structure):
    _fields_ = [("iters", C.c_int32), ("tenure", C.c_int32), ("accept_worsening", C.c_int32),
                ("eval_mode", C.c_int32), ("nthreads", C.c_int32), ("t0", C.c_int32),
                ("expiry_in", C.POINTER(C.c_int32)), ("best_in", C.POINTER(C.c_int32)),
                ("best_cov_in", C.c_int64), ("best_dist_in", C.c_int64),
                ("best_iter_in", C.c_int32),
                ("n_moves", C.c_int32), ("best_iter", C.c_int32),
                ("best_cov", C.c_int64), ("best_dist", C.c_int64),
                ("final_cov", C.c_int64), ("final_dist", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB_OVERRIDE loads a deliberately mutated copy (mutation tests only)
        path = os.environ.get("ORACLE_LIB_OVERRIDE") or build()
        L = C.CDLL(path)
        i32, i64, p = C.c_int32, C.c_int64, C.c_void_p
        L.oracle_leg.restype = i32
        L.oracle_leg.argtypes = [i32, i32, i32, i32]
        L.oracle_mission_cost.restype = i32
        L.oracle_mission_cost.argtypes = [p, p, p, i32, i32]
        L.oracle_cost_table.restype = None
        L.oracle_cost_table.argtypes = [i32, i32, p, p, p, p, i32]
        L.oracle_cost_table_metric.restype = None
        L.oracle_cost_table_metric.argtypes = [i32, i32, p, p, p, p, i32, i32]
        L.oracle_leg_haversine.restype = i32
        L.oracle_leg_haversine.argtypes = [i32, i32, i32, i32]
        L.oracle_evaluate.restype = None
        L.oracle_evaluate.argtypes = [i32, i32, p, i32, p, i32, p, p]
        L.oracle_rank.restype = i32
        L.oracle_rank.argtypes = [i32, i32, p, p, i32, p, p]
        L.oracle_best_two.restype = None
        L.oracle_best_two.argtypes = [i32, i32, p, i32, p, p, p, p, p]
        L.oracle_swap_full.restype = None
        L.oracle_swap_full.argtypes = [i32, i32, p, i32, p, i32, i32, i32, p, p]
        L.oracle_swap_best_two.restype = None
        L.oracle_swap_best_two.argtypes = [i32, i32, p, i32, p, i32, i32, i32, p, p]
        L.oracle_swap_table.restype = None
        L.oracle_swap_table.argtypes = [i32, i32, p, p, i32, p, i32, p, p, i32]
        L.oracle_tabu.restype = i32
        L.oracle_tabu.argtypes = [i32, i32, p, p, i32, i32, p, C.POINTER(TabuIO), p, p, p, p]
        L.oracle_bruteforce.restype = i64
        L.oracle_bruteforce.argtypes = [i32, i32, p, p, i32, i32, p, p, p]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def leg(x1: int, y1: int, x2: int, y2: int) -> int:
    return int(lib().oracle_leg(x1, y1, x2, y2))


def cost_table(base_xy, pick_xy, drop_xy, nthreads: int = 1, haversine: bool = False) -> np.ndarray:
    """B x M int32 round-trip cost table; haversine: coordinates are (latitude,
    longitude) microdegrees and the legs follow Eq. 1."""
    bx, px, dx = _i32(base_xy), _i32(pick_xy), _i32(drop_xy)
    B, M = bx.shape[0], px.shape[0]
    out = np.empty((B, M), dtype=np.int32)
    lib().oracle_cost_table_metric(B, M, _p(bx), _p(px), _p(dx), _p(out), nthreads, 1 if haversine else 0)
    return out


def leg_haversine(lat1: int, lon1: int, lat2: int, lon2: int) -> int:
    return int(lib().oracle_leg_haversine(lat1, lon1, lat2, lon2))


def evaluate(cost: np.ndarray, open_, R: int):
    cost = _i32(cost)
    o = _i32(open_)
    c, d = C.c_int64(), C.c_int64()
    lib().oracle_evaluate(cost.shape[0], cost.shape[1], _p(cost), o.size, _p(o), R,
                          C.byref(c), C.byref(d))
    return int(c.value), int(d.value)


def rank(cost: np.ndarray, K: int, avail=None):
    cost = _i32(cost)
    B, M = cost.shape
    out = np.empty(K, dtype=np.int32)
    rs = np.empty(B, dtype=np.int64)
    av = None if avail is None else np.ascontiguousarray(avail, dtype=np.uint8)
    rc = lib().oracle_rank(B, M, _p(cost), _p(av), K, _p(out), _p(rs))
    if rc != 0:
        raise ValueError("fewer than K available bases")
    return out, rs


def best_two(cost: np.ndarray, open_):
    cost = _i32(cost)
    o = _i32(open_)
    B, M = cost.shape
    a, b, b1, b2 = (np.empty(M, dtype=np.int32) for _ in range(4))
    lib().oracle_best_two(B, M, _p(cost), o.size, _p(o), _p(a), _p(b), _p(b1), _p(b2))
    return a, b, b1, b2


def swap_full(cost, open_, R, i, j):
    cost, o = _i32(cost), _i32(open_)
    c, d = C.c_int64(), C.c_int64()
    lib().oracle_swap_full(cost.shape[0], cost.shape[1], _p(cost), o.size, _p(o), R, i, j,
                           C.byref(c), C.byref(d))
    return int(c.value), int(d.value)


def swap_best_two(cost, open_, R, i, j):
    cost, o = _i32(cost), _i32(open_)
    c, d = C.c_int64(), C.c_int64()
    lib().oracle_swap_best_two(cost.shape[0], cost.shape[1], _p(cost), o.size, _p(o), R, i, j,
                               C.byref(c), C.byref(d))
    return int(c.value), int(d.value)


def swap_table(cost, open_, R, avail=None, nthreads: int = 1):
    """F(i, j) for every open i and closed available j, as two B x B arrays
    (covered count, distance); entries of other pairs are set to -1."""
    cost, o = _i32(cost), _i32(open_)
    B, M = cost.shape
    fc = np.full((B, B), -1, dtype=np.int64)
    fd = np.full((B, B), -1, dtype=np.int64)
    av = None if avail is None else np.ascontiguousarray(avail, dtype=np.uint8)
    lib().oracle_swap_table(B, M, _p(cost), _p(av), o.size, _p(o), R, _p(fc), _p(fd), nthreads)
    return fc, fd


@dataclass
class TabuResult:
    moves: list            # list of (iter, i, j, flags, cov, dist)
    best_open: np.ndarray  # best placement, sorted ascending
    best_cov: int
    best_dist: int
    best_iter: int
    final_open: np.ndarray  # sorted ascending
    final_cov: int
    final_dist: int
    expiry: np.ndarray


def tabu(cost, K, R, iters, tenure, start_open=None, avail=None, accept_worsening=True,
         eval_mode: int = 0, nthreads: int = 1, t0: int = 0, expiry_in=None, best_in=None,
         best_cov_in: int = 0, best_dist_in: int = 0, best_iter_in: int = -1) -> TabuResult:
    """Tabu search (Alg. 3 as read for identical vehicles) from start_open (default: ranking)."""
    cost = _i32(cost)
    B, M = cost.shape
    if start_open is None:
        start_open, _ = rank(cost, K, avail)
    so = _i32(start_open)
    av = None if avail is None else np.ascontiguousarray(avail, dtype=np.uint8)
    io = TabuIO()
    io.iters, io.tenure = iters, tenure
    io.accept_worsening = 1 if accept_worsening else 0
    io.eval_mode, io.nthreads, io.t0 = eval_mode, nthreads, t0
    keep = []
    if expiry_in is not None:
        e = _i32(expiry_in)
        keep.append(e)
        io.expiry_in = e.ctypes.data_as(C.POINTER(C.c_int32))
    if best_in is not None:
        bi = _i32(best_in)
        keep.append(bi)
        io.best_in = bi.ctypes.data_as(C.POINTER(C.c_int32))
        io.best_cov_in, io.best_dist_in, io.best_iter_in = best_cov_in, best_dist_in, best_iter_in
    traj = (Move * max(1, iters))()
    best_open = np.empty(K, dtype=np.int32)
    final_open = np.empty(K, dtype=np.int32)
    expiry = np.empty(B, dtype=np.int32)
    lib().oracle_tabu(B, M, _p(cost), _p(av), K, R, _p(so), C.byref(io), C.cast(traj, C.c_void_p),
                      _p(best_open), _p(final_open), _p(expiry))
    moves = [(traj[k].iter, traj[k].i, traj[k].j, traj[k].flags, traj[k].cov, traj[k].dist)
             for k in range(io.n_moves)]
    return TabuResult(moves, np.sort(best_open), io.best_cov, io.best_dist, io.best_iter,
                      np.sort(final_open), io.final_cov, io.final_dist, expiry)


@dataclass
class LocalSearchResult:
    moves: list             # list of (move number, i, j, MOVE_NEW_BEST, cov, dist)
    final_open: np.ndarray  # sorted ascending
    final_cov: int
    final_dist: int
    passes: int             # passes started
    local_optimum: bool     # the last pass found no improving swap


def local_search(cost, K, R, perm_slots, perm_cands, start_open=None, avail=None, max_moves: int = 100000,
                 eval_mode: str = "table", nthreads: int = 1) -> LocalSearchResult:
    """Local search (Alg. 2, Sec. 4.2) read for identical vehicles.

    The moves are base swaps.  The closed available bases sit at candidate
    positions 0 .. nC-1 (ascending ids at the start); closing the base of slot
    s and opening the base at position c puts the closed base at position c.
    Pass p visits the K x nC (slot, position) pairs with the slot loop outside,
    in the orders perm_slots[p] and perm_cands[p] (the paper's two random
    permutations, here supplied); every pair is judged against the current
    placement and the first strictly better one (more covered, then less
    distance) is applied on the spot, the scan going on with the next pair.
    A pass that moved is followed by the next pass; a pass that did not ends
    the search at a local optimum.  The search also ends when the passes or
    max_moves run out.

    eval_mode "full" judges each pair by evaluating the swapped placement from
    scratch (the plain definition); "table" reads the pair from swap_table of
    the current placement, computed again after every applied move."""
    cost = _i32(cost)
    B, M = cost.shape
    if start_open is None:
        start_open, _ = rank(cost, K, avail)
    O = [int(x) for x in start_open]
    av = np.ones(B, dtype=bool) if avail is None else np.asarray(avail).astype(bool)
    opened = set(O)
    cand = [b for b in range(B) if av[b] and b not in opened]
    nC = len(cand)
    cur = evaluate(cost, O, R)
    moves = []
    if nC == 0:
        return LocalSearchResult(moves, np.sort(np.array(O, dtype=np.int32)), cur[0], cur[1], 0, True)

    def better(x, y):
        return x[0] > y[0] or (x[0] == y[0] and x[1] < y[1])

    passes, optimum = 0, False
    for p in range(len(perm_slots)):
        passes += 1
        pa, pb = perm_slots[p], perm_cands[p]
        moved = False
        table = None
        for u in range(K * nC):
            if len(moves) >= max_moves:
                break
            s, c = int(pa[u // nC]), int(pb[u % nC])
            i, j = O[s], cand[c]
            if eval_mode == "full":
                trial = list(O)
                trial[s] = j
                F = evaluate(cost, trial, R)
            else:
                if table is None:
                    table = swap_table(cost, O, R, avail, nthreads)
                F = (int(table[0][i, j]), int(table[1][i, j]))
            if better(F, cur):
                O[s], cand[c] = j, i
                cur = F
                moves.append((len(moves), i, j, MOVE_NEW_BEST, F[0], F[1]))
                moved = True
                table = None
        if len(moves) >= max_moves:
            break
        if not moved:
            optimum = True
            break
    return LocalSearchResult(moves, np.sort(np.array(O, dtype=np.int32)), cur[0], cur[1], passes, optimum)


def bruteforce(cost, K, R, avail=None):
    """Exact optimum over all K-subsets: (placement, cov, dist, subsets evaluated)."""
    cost = _i32(cost)
    B, M = cost.shape
    out = np.empty(K, dtype=np.int32)
    c, d = C.c_int64(), C.c_int64()
    av = None if avail is None else np.ascontiguousarray(avail, dtype=np.uint8)
    n = lib().oracle_bruteforce(B, M, _p(cost), _p(av), K, R, _p(out), C.byref(c), C.byref(d))
    return out, int(c.value), int(d.value), int(n)
