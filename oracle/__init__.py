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


def forced_moves(cost, open_, R, avail, t, tenure, expiry):
    """Reading A15 (an open base that became unavailable, serving): each
    unavailable open base i, in ascending id, is closed by opening the
    available closed base j with the best objective F(O - i + j) -- more
    covered, then less distance, then the lower j -- tabu ignored.  A forced
    move takes no iteration; both bases get expiry t + tenure (tabu for the
    next `tenure` iterations from t).  Returns (placement in slot order,
    expiry, [(i, j, cov, dist)])."""
    cost = _i32(cost)
    B = cost.shape[0]
    av = np.asarray(avail).astype(bool)
    O = [int(x) for x in open_]
    exp = np.array(expiry, dtype=np.int64).copy()
    done = []
    while True:
        out = sorted(b for b in O if not av[b])
        if not out:
            return O, exp, done
        i = out[0]
        k = O.index(i)
        best = None
        for j in range(B):
            if not av[j] or j in O:
                continue
            trial = O[:k] + [j] + O[k + 1:]
            cov, dist = evaluate(cost, trial, R)
            key = (-cov, dist, j)
            if best is None or key < best[0]:
                best = (key, j, cov, dist)
        if best is None:
            raise ValueError("no available closed base for a forced move")
        _, j, cov, dist = best
        O[k] = j
        exp[i] = exp[j] = t + tenure
        done.append((i, j, cov, dist))


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


def fleet_rank(cost, helipad, K_rotary, K_fixed, avail=None):
    """Alg. 1 with the helipad rule (lines 14-16) and the vehicle assignment of
    lines 20-21: bases by (row sum over every mission, id); a helipad is taken
    only while fewer than K_rotary are taken, until K_rotary + K_fixed bases;
    helipads get rotary-wing vehicles first, then the best-ranked aerodromes;
    the other aerodromes get the fixed-wing vehicles.  Returns (rotary, fixed)."""
    cost = _i32(cost)
    B = cost.shape[0]
    S = cost.astype(np.int64).sum(axis=1)
    av = np.ones(B, dtype=bool) if avail is None else np.asarray(avail).astype(bool)
    order = sorted((b for b in range(B) if av[b]), key=lambda b: (int(S[b]), b))
    chosen, nh = [], 0
    for b in order:
        if len(chosen) == K_rotary + K_fixed:
            break
        if helipad[b]:
            if nh < K_rotary:
                chosen.append(b)
                nh += 1
        else:
            chosen.append(b)
    rot = [b for b in chosen if helipad[b]]
    aer = [b for b in chosen if not helipad[b]]
    rot += aer[:K_rotary - len(rot)]
    fix = aer[K_rotary - nh:]
    if len(rot) != K_rotary or len(fix) != K_fixed:
        raise ValueError("too few available aerodromes for the fixed-wing vehicles")
    return rot, fix


@dataclass
class FleetResult:
    moves: list             # list of (iter, i, j, flags, cov, dist)
    best_rotary: np.ndarray
    best_fixed: np.ndarray
    best_cov: int
    best_dist: int
    best_iter: int
    final_rotary: np.ndarray
    final_fixed: np.ndarray
    final_cov: int
    final_dist: int


def fleet_tabu(cost, helipad, mission_rotary, K_rotary, K_fixed, R, iters, tenure, start_rotary=None,
               start_fixed=None, avail=None, accept_worsening=True, eval_mode: str = "full",
               nthreads: int = 1) -> FleetResult:
    """Tabu search (Alg. 3) with a heterogeneous fleet (Sec. 3, Eq. 6-10, as read):
    rotary-wing vehicles at any base, fixed-wing vehicles at aerodromes only,
    rotary-only missions flown by rotary-wing vehicles only, every mission from
    its nearest compatible open base; the objective is Eq. 2 with coverage.  A
    move takes one vehicle from base i to a closed available base j (an
    aerodrome for a fixed-wing vehicle); tabu expiries, aspiration, fallback,
    the (covered desc, distance asc, i asc, j asc) order and the improving-only
    rule are those of tabu().

    eval_mode "full" evaluates every move's placement from scratch; "table"
    reads the two fast-interchange tables (missions of either type with every
    vehicle, rotary-only missions with the rotary-wing vehicles)."""
    cost = _i32(cost)
    B, M = cost.shape
    heli = np.asarray(helipad).astype(bool)
    rmask = np.asarray(mission_rotary).astype(bool)
    av = np.ones(B, dtype=bool) if avail is None else np.asarray(avail).astype(bool)
    c0 = np.ascontiguousarray(cost[:, ~rmask])
    c1 = np.ascontiguousarray(cost[:, rmask])
    if start_rotary is None and start_fixed is None:
        start_rotary, start_fixed = fleet_rank(cost, heli, K_rotary, K_fixed, avail)
    rot = [int(x) for x in (start_rotary if start_rotary is not None else [])]
    fix = [int(x) for x in (start_fixed if start_fixed is not None else [])]

    def F(r, f):
        a = evaluate(c0, r + f, R) if c0.shape[1] else (0, 0)
        b = evaluate(c1, r, R) if (c1.shape[1] and r) else (0, 0)
        return a[0] + b[0], a[1] + b[1]

    def better(x, y):
        return x[0] > y[0] or (x[0] == y[0] and x[1] < y[1])

    cur = F(rot, fix)
    best, best_iter = cur, -1
    best_r, best_f = list(rot), list(fix)
    expiry = np.zeros(B, dtype=np.int64)
    moves = []
    for t in range(iters):
        opened = set(rot) | set(fix)
        cands = [j for j in range(B) if av[j] and j not in opened]
        if eval_mode == "table":
            t0 = swap_table(c0, rot + fix, R, avail, nthreads) if c0.shape[1] else None
            t1 = swap_table(c1, rot, R, avail, nthreads) if (c1.shape[1] and rot) else None
            v1 = evaluate(c1, rot, R) if (c1.shape[1] and rot) else (0, 0)
        keys = []   # (key for sorting, cov, dist, i, j, kind, slot)
        for kind, group in ((0, rot), (1, fix)):
            for sl, i in enumerate(group):
                for j in cands:
                    if kind == 1 and heli[j]:
                        continue
                    if eval_mode == "table":
                        a = (int(t0[0][i, j]), int(t0[1][i, j])) if t0 is not None else (0, 0)
                        b = ((int(t1[0][i, j]), int(t1[1][i, j])) if t1 is not None else (0, 0)) if kind == 0 else v1
                        f = (a[0] + b[0], a[1] + b[1])
                    else:
                        r2, f2 = list(rot), list(fix)
                        (r2 if kind == 0 else f2)[sl] = j
                        f = F(r2, f2)
                    tabu = t < expiry[i] or t < expiry[j]
                    keys.append(((-f[0], f[1], i, j), f, i, j, kind, sl, tabu))
        if not keys:
            break
        keys.sort(key=lambda k: k[0])
        adm = [k for k in keys if not k[6] or better(k[1], best)]
        pick = adm[0] if adm else keys[0]
        flags = (MOVE_ASPIRATION if pick[6] else 0) if adm else MOVE_FALLBACK
        if not accept_worsening and not better(pick[1], cur):
            break
        _, f, i, j, kind, sl, _ = pick
        (rot if kind == 0 else fix)[sl] = j
        expiry[i] = expiry[j] = t + tenure + 1
        cur = f
        if better(f, best):
            best, best_iter = f, t
            best_r, best_f = list(rot), list(fix)
            flags |= MOVE_NEW_BEST
        moves.append((t, i, j, flags, f[0], f[1]))
    return FleetResult(moves, np.sort(np.array(best_r, dtype=np.int32)), np.sort(np.array(best_f, dtype=np.int32)),
                       best[0], best[1], best_iter, np.sort(np.array(rot, dtype=np.int32)),
                       np.sort(np.array(fix, dtype=np.int32)), cur[0], cur[1])


def bruteforce(cost, K, R, avail=None):
    """Exact optimum over all K-subsets: (placement, cov, dist, subsets evaluated)."""
    cost = _i32(cost)
    B, M = cost.shape
    out = np.empty(K, dtype=np.int32)
    c, d = C.c_int64(), C.c_int64()
    av = None if avail is None else np.ascontiguousarray(avail, dtype=np.uint8)
    n = lib().oracle_bruteforce(B, M, _p(cost), _p(av), K, R, _p(out), C.byref(c), C.byref(d))
    return out, int(c.value), int(d.value), int(n)
