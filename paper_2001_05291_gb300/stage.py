"""Python binding of the staging engine's C ABI (include/stage.h), via ctypes.

Argument marshalling only: every step of the method runs in the engine's CUDA
kernels.  PyTorch supplies device memory (the caching allocator, through the
engine's allocator hook) and the CUDA stream.  There is no CPU fallback: if the
shared library is missing or no GPU is present, the calls raise.

The module-level functions carry the C names (stage_create, stage_load_instance,
stage_rank_bases, stage_evaluate_placement, stage_evaluate_swaps,
stage_tabu_run, ...); ``Context`` wraps the same calls as methods.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libstage.so")

STAGE_OK, STAGE_PENDING = 0, 1
ERRORS = {-1: "INVALID_ARG", -2: "OUT_OF_RANGE", -3: "NO_MEMORY", -4: "ADMISSION", -5: "TIMEOUT",
          -6: "CUDA", -7: "INTERNAL", -8: "NOT_FOUND"}
STAGE_THREADSAFE, STAGE_PROFILE, STAGE_AUTOTUNE, STAGE_FULL_PASS, STAGE_INCREMENTAL = 1, 2, 4, 8, 16
STAGE_NO_PERSIST = 32
STAGE_DESC_DEVICE, STAGE_DESC_HAVERSINE = 1, 2
MOVE_FALLBACK, MOVE_ASPIRATION, MOVE_NEW_BEST = 1, 2, 4
MAX_COORD, MAX_BASES, MAX_MISSIONS, MAX_K = 1 << 24, 65535, 1 << 24, 1024

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class StageConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("flags", C.c_uint32), ("hbm_budget_bytes", C.c_uint64),
                ("max_slots", C.c_int32), ("reserved0", C.c_int32), ("spin_limit", C.c_int64),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("stream", C.c_void_p)]


class StageInstanceDesc(C.Structure):
    _fields_ = [("B", C.c_int32), ("M", C.c_int32), ("flags", C.c_uint32), ("reserved0", C.c_int32),
                ("base_xy", C.c_void_p), ("pick_xy", C.c_void_p), ("drop_xy", C.c_void_p),
                ("base_available", C.c_void_p)]


class StageMove(C.Structure):
    _fields_ = [("iter", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("flags", C.c_int32),
                ("cov", C.c_int64), ("dist", C.c_int64)]


_MOVE_DTYPE = np.dtype([("iter", np.int32), ("i", np.int32), ("j", np.int32), ("flags", np.int32),
                        ("cov", np.int64), ("dist", np.int64)])
assert _MOVE_DTYPE.itemsize == C.sizeof(StageMove)


def _moves(traj, n: int) -> list:
    """The first n stage_move records of a ctypes array, as (iter, i, j,
    flags, cov, dist) tuples of Python ints."""
    if traj is None or n <= 0:
        return []
    return np.frombuffer(traj, dtype=_MOVE_DTYPE, count=n).tolist()


def _moves_array(traj, n: int) -> np.ndarray:
    """The first n stage_move records of a ctypes array as a structured numpy
    view (it keeps the array alive)."""
    if traj is None or n <= 0:
        return np.empty(0, dtype=_MOVE_DTYPE)
    return np.frombuffer(traj, dtype=_MOVE_DTYPE, count=n)


class StageTabuState(C.Structure):
    _fields_ = [("t", C.c_int32), ("best_iter", C.c_int32), ("best_cov", C.c_int64),
                ("best_dist", C.c_int64), ("open", C.c_void_p), ("best_open", C.c_void_p),
                ("tabu_expiry", C.c_void_p)]


class StageTabuParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("R", C.c_int32), ("iters", C.c_int32), ("tenure", C.c_int32),
                ("accept_worsening", C.c_int32), ("reserved0", C.c_int32),
                ("start_open", C.c_void_p), ("resume", C.POINTER(StageTabuState))]


class StageLsParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("R", C.c_int32), ("n_passes", C.c_int32), ("max_moves", C.c_int32),
                ("perm_slots", C.c_void_p), ("perm_cands", C.c_void_p), ("start_open", C.c_void_p)]


class StageLsResult(C.Structure):
    _fields_ = [("n_moves", C.c_int32), ("passes", C.c_int32), ("local_optimum", C.c_int32),
                ("reserved0", C.c_int32), ("final_cov", C.c_int64), ("final_dist", C.c_int64),
                ("final_open", C.c_void_p)]


class StageFleetParams(C.Structure):
    _fields_ = [("K_rotary", C.c_int32), ("K_fixed", C.c_int32), ("R", C.c_int32), ("iters", C.c_int32),
                ("tenure", C.c_int32), ("accept_worsening", C.c_int32), ("base_helipad", C.c_void_p),
                ("mission_rotary", C.c_void_p), ("start_rotary", C.c_void_p), ("start_fixed", C.c_void_p)]


class StageFleetResult(C.Structure):
    _fields_ = [("n_moves", C.c_int32), ("best_iter", C.c_int32), ("best_cov", C.c_int64),
                ("best_dist", C.c_int64), ("final_cov", C.c_int64), ("final_dist", C.c_int64),
                ("best_rotary", C.c_void_p), ("best_fixed", C.c_void_p), ("final_rotary", C.c_void_p),
                ("final_fixed", C.c_void_p)]


class StageUpdate(C.Structure):
    _fields_ = [("n_add", C.c_int32), ("n_remove", C.c_int32), ("n_unavail", C.c_int32),
                ("n_avail", C.c_int32), ("add_pick_xy", C.c_void_p), ("add_drop_xy", C.c_void_p),
                ("remove_ids", C.c_void_p), ("unavail_ids", C.c_void_p), ("avail_ids", C.c_void_p)]


class StageRequest(C.Structure):
    _fields_ = [("inst", C.c_uint64), ("desc", C.POINTER(StageInstanceDesc)),
                ("update", C.POINTER(StageUpdate)), ("params", StageTabuParams),
                ("traj", C.c_void_p), ("best_open", C.c_void_p), ("final_open", C.c_void_p),
                ("resume_resident", C.c_int32), ("reserved1", C.c_int32)]


class StageResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_moves", C.c_int32), ("best_iter", C.c_int32),
                ("n_forced", C.c_int32), ("best_cov", C.c_int64), ("best_dist", C.c_int64),
                ("final_cov", C.c_int64), ("final_dist", C.c_int64), ("t_submit_ns", C.c_int64),
                ("t_start_ns", C.c_int64), ("t_end_ns", C.c_int64)]


class StageTabuResult(C.Structure):
    _fields_ = [("n_moves", C.c_int32), ("best_iter", C.c_int32), ("best_cov", C.c_int64),
                ("best_dist", C.c_int64), ("final_cov", C.c_int64), ("final_dist", C.c_int64),
                ("best_open", C.c_void_p), ("final_open", C.c_void_p),
                ("end_state", C.POINTER(StageTabuState))]


_lib = None


def lib():
    """The loaded engine library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"the CUDA engine library is missing ({LIB_PATH}); "
                               "build it with paper_2001_05291_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        i32, i64, p, st = C.c_int32, C.c_int64, C.c_void_p, C.c_int32
        sig = {
            "stage_create": ([C.POINTER(StageConfig), C.POINTER(p)], st),
            "stage_destroy": ([p], st),
            "stage_last_error": ([p, C.c_char_p, C.c_size_t], st),
            "stage_version": ([], i32),
            "stage_memory_used": ([p, C.POINTER(C.c_uint64)], st),
            "stage_load_instance": ([p, C.POINTER(StageInstanceDesc), C.POINTER(C.c_uint64)], st),
            "stage_unload_instance": ([p, C.c_uint64], st),
            "stage_rank_bases": ([p, C.c_uint64, i32, p, p], st),
            "stage_evaluate_placement": ([p, C.c_uint64, p, i32, i32, C.POINTER(i64), C.POINTER(i64)], st),
            "stage_evaluate_swaps": ([p, C.c_uint64, p, i32, i32, p, p], st),
            "stage_tabu_run": ([p, C.c_uint64, C.POINTER(StageTabuParams), C.POINTER(StageTabuResult), p], st),
            "stage_tabu_batch": ([p, i32, C.POINTER(C.c_uint64), C.POINTER(StageTabuParams),
                                  C.POINTER(StageTabuResult), C.POINTER(p)], st),
            "stage_local_search": ([p, C.c_uint64, C.POINTER(StageLsParams), C.POINTER(StageLsResult), p], st),
            "stage_fleet_tabu": ([p, C.c_uint64, C.POINTER(StageFleetParams), C.POINTER(StageFleetResult), p], st),
            "stage_kernel_stats": ([p, C.c_char_p, C.POINTER(i64), C.POINTER(C.c_double)], st),
            "stage_reset_stats": ([p], st),
            "stage_read_table": ([p, C.c_uint64, i32, i32, i32, i32, p], st),
            "stage_best_two": ([p, C.c_uint64, p, i32, i32, i32, i32, p, p, p, p], st),
            "stage_autotune": ([p, C.c_uint64, p, i32, i32, C.POINTER(i32)], st),
            "stage_update_instance": ([p, C.c_uint64, C.POINTER(StageUpdate)], st),
            "stage_batch_submit": ([p, C.POINTER(StageRequest), i32, C.POINTER(C.c_uint64)], st),
            "stage_poll": ([p, C.c_uint64, C.POINTER(StageResult), i32], st),
            "stage_test_wait_timeout": ([p], st),
            "stage_test_batch_schedule": ([i32, p, p, i32, p, p, C.POINTER(C.c_double)], st),
            "stage_evaluate_swaps_noalloc": ([p, i32, i32, i32, p, p, i32, i32, p, p, p, C.c_char_p,
                                              C.c_size_t], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class StageError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{ERRORS.get(status, status)}: {message}")
        self.status = status
        self.message = message


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _host_i32(a, n=None) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a), dtype=np.int32)
    if n is not None and out.size != n:
        raise ValueError(f"expected {n} values, got {out.size}")
    return out


class TabuResult:
    """A Tabu search's result.  moves_array: the applied moves as a numpy
    structured array (iter, i, j, flags, cov, dist), a view of the returned
    trajectory; moves: the same as a list of tuples of Python ints, built from
    it on first use."""

    def __init__(self, n_moves, best_open, best_cov, best_dist, best_iter, final_open, final_cov, final_dist,
                 moves=None, end_state=None):
        self.n_moves, self.best_open, self.best_cov, self.best_dist = n_moves, best_open, best_cov, best_dist
        self.best_iter, self.final_open, self.final_cov, self.final_dist = best_iter, final_open, final_cov, final_dist
        self.end_state = end_state
        if isinstance(moves, np.ndarray):
            self.moves_array, self._moves = moves, None
        else:
            self.moves_array, self._moves = None, list(moves) if moves is not None else []

    @property
    def moves(self) -> list:
        if self._moves is None:
            self._moves = self.moves_array.tolist()
        return self._moves

    def __repr__(self):
        return (f"TabuResult(n_moves={self.n_moves}, best_cov={self.best_cov}, best_dist={self.best_dist}, "
                f"best_iter={self.best_iter}, final_cov={self.final_cov}, final_dist={self.final_dist})")


@dataclass
class FleetResult:
    n_moves: int
    best_rotary: np.ndarray
    best_fixed: np.ndarray
    best_cov: int
    best_dist: int
    best_iter: int
    final_rotary: np.ndarray
    final_fixed: np.ndarray
    final_cov: int
    final_dist: int
    moves: list = field(default_factory=list)   # (iter, i, j, flags, cov, dist)


@dataclass
class LocalSearchResult:
    n_moves: int
    passes: int
    local_optimum: bool
    final_open: np.ndarray
    final_cov: int
    final_dist: int
    moves: list = field(default_factory=list)   # (move number, i, j, flags, cov, dist)


class _TorchAllocator:
    """Backs the engine's device allocations with PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=f"cuda:{self.device}")
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, nbytes, user):
        self.live.pop(ptr, None)


class Context:
    """One engine context on one GPU (stage_create / stage_destroy)."""

    def __init__(self, device: int = 0, profile: bool = False, threadsafe: bool = False,
                 hbm_budget: int = 0, max_slots: int = 0, spin_limit: int = 0,
                 torch_memory: bool = True, stream=None, autotune: bool = False, full_pass: bool = False,
                 incremental: bool = False, persist: bool = True, allocator=None):
        L = lib()
        cfg = StageConfig()
        cfg.device = device
        cfg.flags = ((STAGE_PROFILE if profile else 0) | (STAGE_THREADSAFE if threadsafe else 0) |
                     (STAGE_AUTOTUNE if autotune else 0) | (STAGE_FULL_PASS if full_pass else 0) |
                     (STAGE_INCREMENTAL if incremental else 0) | (0 if persist else STAGE_NO_PERSIST))
        cfg.hbm_budget_bytes = hbm_budget
        cfg.max_slots = max_slots
        cfg.spin_limit = spin_limit
        self._alloc = None
        self.torch_stream = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise StageError(-6, "no CUDA device")
            # allocator: an object with alloc_cb / free_cb (ALLOC_FN / FREE_FN
            # callbacks); default: PyTorch's caching allocator
            self._alloc = allocator if allocator is not None else _TorchAllocator(device)
            cfg.alloc = self._alloc.alloc_cb
            cfg.free = self._alloc.free_cb
            self.torch_stream = stream if stream is not None else torch.cuda.Stream(device=device)
            cfg.stream = self.torch_stream.cuda_stream
        elif stream is not None:
            cfg.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = C.c_void_p()
        rc = L.stage_create(C.byref(cfg), C.byref(h))
        if rc != STAGE_OK:
            raise StageError(rc, "stage_create failed")
        self._h = h
        self._cfg = cfg
        self.device = device

    # ------------------------------------------------------------- plumbing
    def _check(self, rc: int):
        if rc < 0:
            buf = C.create_string_buffer(512)
            lib().stage_last_error(self._h, buf, 512)
            raise StageError(rc, buf.value.decode(errors="replace"))
        return rc

    def close(self):
        if getattr(self, "_h", None):
            lib().stage_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory_used(self) -> int:
        v = C.c_uint64()
        self._check(lib().stage_memory_used(self._h, C.byref(v)))
        return int(v.value)

    def test_wait_timeout(self):
        """stage_test_wait_timeout: one bounded device wait on a flag nothing
        sets; raises StageError (TIMEOUT) when it gives up, as expected."""
        self._check(lib().stage_test_wait_timeout(self._h))

    # ------------------------------------------------------------- instances
    def load_instance(self, base_xy, pick_xy, drop_xy, base_available=None, haversine: bool = False) -> int:
        """stage_load_instance.  numpy arrays are copied from the host; CUDA
        tensors (int32, contiguous) are read on the device.  haversine: the
        coordinates are (latitude, longitude) microdegrees (Eq. 1 legs)."""
        d = StageInstanceDesc()
        keep = []
        if _is_cuda_tensor(base_xy):
            for t in (base_xy, pick_xy, drop_xy):
                if not _is_cuda_tensor(t) or t.dtype.itemsize != 4 or not t.is_contiguous():
                    raise ValueError("device inputs must all be contiguous int32 CUDA tensors")
            d.B, d.M = base_xy.numel() // 2, pick_xy.numel() // 2
            d.flags = STAGE_DESC_DEVICE
            d.base_xy, d.pick_xy, d.drop_xy = base_xy.data_ptr(), pick_xy.data_ptr(), drop_xy.data_ptr()
            if base_available is not None:
                d.base_available = base_available.data_ptr()
            keep = [base_xy, pick_xy, drop_xy, base_available]
        else:
            b, p, q = (_host_i32(x) for x in (base_xy, pick_xy, drop_xy))
            d.B, d.M = b.size // 2, p.size // 2
            d.base_xy, d.pick_xy, d.drop_xy = _ptr(b), _ptr(p), _ptr(q)
            keep = [b, p, q]
            if base_available is not None:
                av = np.ascontiguousarray(base_available, dtype=np.uint8)
                d.base_available = _ptr(av)
                keep.append(av)
        if haversine:
            d.flags |= STAGE_DESC_HAVERSINE
        h = C.c_uint64()
        self._check(lib().stage_load_instance(self._h, C.byref(d), C.byref(h)))
        del keep
        return int(h.value)

    def unload_instance(self, inst: int):
        self._check(lib().stage_unload_instance(self._h, inst))

    def rank_bases(self, inst: int, K: int, B: int | None = None, rowsum: bool = True):
        out = np.empty(K, dtype=np.int32)
        rs = np.empty(B, dtype=np.int64) if (rowsum and B) else None
        self._check(lib().stage_rank_bases(self._h, inst, K, _ptr(out), None if rs is None else _ptr(rs)))
        return out, rs

    def evaluate_placement(self, inst: int, open_, R: int):
        o = _host_i32(open_)
        cov, dist = C.c_int64(), C.c_int64()
        self._check(lib().stage_evaluate_placement(self._h, inst, _ptr(o), o.size, R,
                                                   C.byref(cov), C.byref(dist)))
        return int(cov.value), int(dist.value)

    def evaluate_swaps(self, inst: int, open_, R: int, B: int):
        o = _host_i32(open_)
        fc = np.empty(o.size * B, dtype=np.int64)
        fd = np.empty(o.size * B, dtype=np.int64)
        self._check(lib().stage_evaluate_swaps(self._h, inst, _ptr(o), o.size, R, _ptr(fc), _ptr(fd)))
        return fc.reshape(o.size, B), fd.reshape(o.size, B)

    def fleet_tabu(self, inst: int, K_rotary: int, K_fixed: int, R: int, iters: int, tenure: int, base_helipad,
                   mission_rotary, start_rotary=None, start_fixed=None, accept_worsening: bool = True,
                   trajectory: bool = True) -> FleetResult:
        """stage_fleet_tabu: rotary- and fixed-wing vehicles, helipads, rotary-only missions."""
        p = StageFleetParams()
        p.K_rotary, p.K_fixed, p.R, p.iters, p.tenure = K_rotary, K_fixed, R, iters, tenure
        p.accept_worsening = 1 if accept_worsening else 0
        hp = np.ascontiguousarray(base_helipad, dtype=np.uint8)
        mr = np.ascontiguousarray(mission_rotary, dtype=np.uint8)
        p.base_helipad, p.mission_rotary = _ptr(hp), _ptr(mr)
        keep = [hp, mr]
        if start_rotary is not None or start_fixed is not None:
            sr = _host_i32(start_rotary if start_rotary is not None else [], K_rotary)
            sf = _host_i32(start_fixed if start_fixed is not None else [], K_fixed)
            keep += [sr, sf]
            p.start_rotary = _ptr(sr) if K_rotary else None
            p.start_fixed = _ptr(sf) if K_fixed else None
            if not K_rotary and not K_fixed:
                raise ValueError("no vehicles")
            if p.start_rotary is None and p.start_fixed is None:
                raise ValueError("start given for zero vehicles")
        r = StageFleetResult()
        br, bf = np.empty(K_rotary, dtype=np.int32), np.empty(K_fixed, dtype=np.int32)
        fr, ff = np.empty(K_rotary, dtype=np.int32), np.empty(K_fixed, dtype=np.int32)
        r.best_rotary, r.best_fixed = _ptr(br), _ptr(bf)
        r.final_rotary, r.final_fixed = _ptr(fr), _ptr(ff)
        traj = (StageMove * max(1, iters))() if trajectory else None
        self._check(lib().stage_fleet_tabu(self._h, inst, C.byref(p), C.byref(r),
                                           C.cast(traj, C.c_void_p) if traj is not None else None))
        moves = _moves(traj, min(r.n_moves, iters))
        return FleetResult(r.n_moves, br, bf, r.best_cov, r.best_dist, r.best_iter, fr, ff, r.final_cov,
                           r.final_dist, moves)

    def local_search(self, inst: int, K: int, R: int, perm_slots, perm_cands, max_moves: int = 100000,
                     start_open=None, trajectory: bool = True) -> LocalSearchResult:
        """stage_local_search (Alg. 2): perm_slots [passes, K], perm_cands [passes, nC] with
        nC = available bases - K; row p of each is pass p's scan order."""
        ps = np.ascontiguousarray(np.asarray(perm_slots), dtype=np.int32)
        pc = np.ascontiguousarray(np.asarray(perm_cands), dtype=np.int32)
        if ps.ndim != 2 or pc.ndim != 2 or ps.shape[0] != pc.shape[0] or ps.shape[1] != K:
            raise ValueError("perm_slots must be [passes, K] and perm_cands [passes, nC]")
        p = StageLsParams()
        p.K, p.R, p.n_passes, p.max_moves = K, R, ps.shape[0], max_moves
        p.perm_slots, p.perm_cands = _ptr(ps), (_ptr(pc) if pc.size else None)
        keep = [ps, pc]
        if start_open is not None:
            so = _host_i32(start_open, K)
            keep.append(so)
            p.start_open = _ptr(so)
        r = StageLsResult()
        fin = np.empty(K, dtype=np.int32)
        r.final_open = _ptr(fin)
        traj = (StageMove * max(1, max_moves))() if trajectory else None
        self._check(lib().stage_local_search(self._h, inst, C.byref(p), C.byref(r),
                                             C.cast(traj, C.c_void_p) if traj is not None else None))
        moves = _moves(traj, min(r.n_moves, max_moves))
        return LocalSearchResult(r.n_moves, r.passes, bool(r.local_optimum), fin, r.final_cov, r.final_dist,
                                 moves)

    def tabu_run(self, inst: int, K: int, R: int, iters: int, tenure: int, start_open=None,
                 accept_worsening: bool = True, resume: dict | None = None, B: int | None = None,
                 trajectory: bool = True, end_state: bool = False) -> TabuResult:
        p = StageTabuParams()
        p.K, p.R, p.iters, p.tenure = K, R, iters, tenure
        p.accept_worsening = 1 if accept_worsening else 0
        keep = []
        if start_open is not None:
            so = _host_i32(start_open, K)
            keep.append(so)
            p.start_open = _ptr(so)
        if resume is not None:
            rs = StageTabuState()
            ro, rb, re_ = (_host_i32(resume[k]) for k in ("open", "best_open", "tabu_expiry"))
            keep += [ro, rb, re_]
            rs.t, rs.best_iter = resume["t"], resume["best_iter"]
            rs.best_cov, rs.best_dist = resume["best_cov"], resume["best_dist"]
            rs.open, rs.best_open, rs.tabu_expiry = _ptr(ro), _ptr(rb), _ptr(re_)
            keep.append(rs)
            p.resume = C.pointer(rs)
        r = StageTabuResult()
        best = np.empty(K, dtype=np.int32)
        fin = np.empty(K, dtype=np.int32)
        r.best_open, r.final_open = _ptr(best), _ptr(fin)
        es = None
        if end_state:
            if B is None:
                raise ValueError("end_state needs B")
            es_open, es_best, es_exp = (np.empty(K, dtype=np.int32), np.empty(K, dtype=np.int32),
                                        np.empty(B, dtype=np.int32))
            es = StageTabuState()
            es.open, es.best_open, es.tabu_expiry = _ptr(es_open), _ptr(es_best), _ptr(es_exp)
            r.end_state = C.pointer(es)
        traj = (StageMove * max(1, iters))() if trajectory else None
        self._check(lib().stage_tabu_run(self._h, inst, C.byref(p), C.byref(r),
                                         C.cast(traj, C.c_void_p) if traj is not None else None))
        moves = _moves_array(traj, min(r.n_moves, iters))
        out = TabuResult(r.n_moves, best, r.best_cov, r.best_dist, r.best_iter, fin, r.final_cov,
                         r.final_dist, moves)
        if es is not None:
            out.end_state = dict(t=es.t, best_iter=es.best_iter, best_cov=es.best_cov,
                                 best_dist=es.best_dist, open=es_open, best_open=es_best,
                                 tabu_expiry=es_exp)
        return out

    def tabu_batch(self, requests, trajectory: bool = True) -> list:
        """stage_tabu_batch: many Tabu searches in one launch.  Each request is a
        dict(inst, K, R, iters, tenure[, start_open][, accept_worsening]); returns
        one TabuResult per request, in order."""
        n = len(requests)
        hs = (C.c_uint64 * max(1, n))()
        ps = (StageTabuParams * max(1, n))()
        rs = (StageTabuResult * max(1, n))()
        tp = (C.c_void_p * max(1, n))()
        keep, outs = [], []
        for k, q in enumerate(requests):
            hs[k] = q["inst"]
            P = ps[k]
            P.K, P.R, P.iters, P.tenure = q["K"], q["R"], q["iters"], q["tenure"]
            P.accept_worsening = 1 if q.get("accept_worsening", True) else 0
            if q.get("start_open") is not None:
                so = _host_i32(q["start_open"], q["K"])
                keep.append(so)
                P.start_open = _ptr(so)
            best = np.empty(q["K"], dtype=np.int32)
            fin = np.empty(q["K"], dtype=np.int32)
            rs[k].best_open, rs[k].final_open = _ptr(best), _ptr(fin)
            traj = (StageMove * max(1, q["iters"]))() if trajectory else None
            tp[k] = C.cast(traj, C.c_void_p) if traj is not None else None
            outs.append((best, fin, traj))
        self._check(lib().stage_tabu_batch(self._h, n, hs, ps, rs, tp))
        results = []
        for k, (best, fin, traj) in enumerate(outs):
            r = rs[k]
            moves = _moves_array(traj, min(r.n_moves, requests[k]["iters"]))
            results.append(TabuResult(r.n_moves, best, r.best_cov, r.best_dist, r.best_iter, fin, r.final_cov,
                                      r.final_dist, moves))
        return results

    def best_two(self, inst: int, open_, R: int, M: int, tabu_steps: int = 0, tenure: int = 0):
        o = _host_i32(open_)
        a, b, b1, b2 = (np.empty(M, dtype=np.int32) for _ in range(4))
        self._check(lib().stage_best_two(self._h, inst, _ptr(o), o.size, R, tabu_steps, tenure,
                                         _ptr(a), _ptr(b), _ptr(b1), _ptr(b2)))
        return a, b, b1, b2

    def read_table(self, inst: int, b0: int, nb: int, m0: int, nm: int) -> np.ndarray:
        out = np.empty((nb, nm), dtype=np.int32)
        self._check(lib().stage_read_table(self._h, inst, b0, nb, m0, nm, _ptr(out)))
        return out

    def update_instance(self, inst: int, add_pick=None, add_drop=None, remove=None, unavailable=None,
                        available=None):
        """stage_update_instance: append missions, withdraw mission ids, close or reopen bases."""
        u, keep = _make_update(add_pick, add_drop, remove, unavailable, available)
        self._check(lib().stage_update_instance(self._h, inst, C.byref(u)))
        del keep

    def batch_submit(self, requests):
        """stage_batch_submit.  Each request is a dict: inst (handle) or base_xy/pick_xy/drop_xy
        (+ base_available) for an instance given by value; K, R, iters, tenure;
        optional start_open, accept_worsening, update (dict of update_instance's arguments),
        resume_resident (continue from the resident instance's kept end state, A15 forced moves
        after an update; the result's n_forced counts them).
        Returns a list of BatchTicket; call .wait() (or Context.poll) for results."""
        n = len(requests)
        arr = (StageRequest * max(1, n))()
        tickets = (C.c_uint64 * max(1, n))()
        keep, outs = [], []
        for k, rq in enumerate(requests):
            r = arr[k]
            if "inst" in rq and rq["inst"]:
                r.inst = rq["inst"]
            else:
                d = StageInstanceDesc()
                b, p, q = (_host_i32(rq[x]) for x in ("base_xy", "pick_xy", "drop_xy"))
                d.B, d.M = b.size // 2, p.size // 2
                d.base_xy, d.pick_xy, d.drop_xy = _ptr(b), _ptr(p), _ptr(q)
                if rq.get("haversine"):
                    d.flags = STAGE_DESC_HAVERSINE
                keep += [b, p, q, d]
                if rq.get("base_available") is not None:
                    av = np.ascontiguousarray(rq["base_available"], dtype=np.uint8)
                    d.base_available = _ptr(av)
                    keep.append(av)
                r.desc = C.pointer(d)
            if rq.get("update"):
                u, kk = _make_update(**rq["update"])
                keep += [u, kk]
                r.update = C.pointer(u)
            K, iters = rq["K"], rq["iters"]
            r.params.K, r.params.R, r.params.iters, r.params.tenure = K, rq["R"], iters, rq["tenure"]
            r.params.accept_worsening = 1 if rq.get("accept_worsening", True) else 0
            r.resume_resident = 1 if rq.get("resume_resident") else 0
            if rq.get("start_open") is not None:
                so = _host_i32(rq["start_open"], K)
                keep.append(so)
                r.params.start_open = _ptr(so)
            traj = (StageMove * max(1, iters))()
            best = np.empty(K, dtype=np.int32)
            fin = np.empty(K, dtype=np.int32)
            r.traj, r.best_open, r.final_open = C.cast(traj, C.c_void_p), _ptr(best), _ptr(fin)
            outs.append((traj, best, fin))
        self._check(lib().stage_batch_submit(self._h, arr, n, tickets))
        del keep
        return [BatchTicket(self, int(tickets[k]), *outs[k]) for k in range(n)]

    def poll(self, ticket: "BatchTicket", timeout_us: int = -1):
        """stage_poll: None while the ticket runs (after waiting up to timeout_us), else its result."""
        res = StageResult()
        rc = lib().stage_poll(self._h, ticket.id, C.byref(res), timeout_us)
        if rc == STAGE_PENDING:
            return None
        ticket.done = True
        if rc < 0:
            buf = C.create_string_buffer(512)
            lib().stage_last_error(self._h, buf, 512)
            raise StageError(rc, f"batch request failed (ticket {ticket.id}); the context's last error: "
                                 f"{buf.value.decode(errors='replace')}")
        moves = _moves_array(ticket.traj, res.n_moves)
        out = TabuResult(res.n_moves, ticket.best, res.best_cov, res.best_dist, res.best_iter, ticket.final,
                         res.final_cov, res.final_dist, moves)
        out.timing = dict(submit_ns=res.t_submit_ns, start_ns=res.t_start_ns, end_ns=res.t_end_ns)
        out.n_forced = res.n_forced
        return out

    def autotune(self, inst: int, K: int, R: int, open_=None) -> int:
        """stage_autotune: measured missions-per-block of the swap pass for this shape."""
        seg = C.c_int32()
        o = None if open_ is None else _host_i32(open_, K)
        self._check(lib().stage_autotune(self._h, inst, None if o is None else _ptr(o), K, R, C.byref(seg)))
        return int(seg.value)

    def kernel_stats(self, name: str):
        n, ms = C.c_int64(), C.c_double()
        self._check(lib().stage_kernel_stats(self._h, name.encode(), C.byref(n), C.byref(ms)))
        return int(n.value), float(ms.value)

    def reset_stats(self):
        self._check(lib().stage_reset_stats(self._h))


class BatchTicket:
    """A submitted batch request; its output buffers live here until collected."""

    def __init__(self, ctx, tid, traj, best, final):
        self.ctx, self.id, self.traj, self.best, self.final = ctx, tid, traj, best, final
        self.done = False

    def wait(self, timeout_us: int = -1):
        return self.ctx.poll(self, timeout_us)


def _make_update(add_pick=None, add_drop=None, remove=None, unavailable=None, available=None):
    u = StageUpdate()
    keep = []
    if (add_pick is None) != (add_drop is None):
        raise ValueError("add_pick and add_drop go together")
    if add_pick is not None:
        ap, ad = _host_i32(add_pick), _host_i32(add_drop)
        if ap.size != ad.size:
            raise ValueError("add_pick and add_drop differ in size")
        if ap.size % 2:
            raise ValueError("add_pick and add_drop hold (x, y) pairs")
        u.n_add, u.add_pick_xy, u.add_drop_xy = ap.size // 2, _ptr(ap), _ptr(ad)
        keep += [ap, ad]
    for name, cnt, ptr in ((remove, "n_remove", "remove_ids"), (unavailable, "n_unavail", "unavail_ids"),
                           (available, "n_avail", "avail_ids")):
        if name is not None:
            a = _host_i32(name)
            setattr(u, cnt, a.size)
            setattr(u, ptr, _ptr(a))
            keep.append(a)
    return u, keep


def evaluate_swaps_noalloc(cost, M: int, open_, R: int, out_cov, out_dist, base_available=None,
                           stream=None):
    """stage_evaluate_swaps_noalloc on CUDA tensors: cost [B, M_pad] int32, open_ [K]
    int32, out_cov / out_dist [K, B] int64, base_available [B] uint8 or None.  For
    callers that cannot allocate device memory; see include/stage.h.  Only
    enqueues on `stream` (a torch stream or raw handle; None = legacy default)."""
    import torch
    tensors = [cost, open_, out_cov, out_dist] + ([] if base_available is None else [base_available])
    for t in tensors:
        if not _is_cuda_tensor(t) or not t.is_contiguous():
            raise ValueError("inputs and outputs must be contiguous CUDA tensors")
    # the scratch address is looked up for the current device, and the kernels
    # run there: every tensor must live on it
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in tensors):
        raise ValueError(f"every tensor must be on the current CUDA device (cuda:{dev})")
    if cost.dim() != 2 or cost.dtype != torch.int32:
        raise ValueError("cost must be a 2-D int32 tensor [B, M_pad]")
    if open_.dtype != torch.int32:
        raise ValueError("open_ must be an int32 tensor")
    if out_cov.dtype != torch.int64 or out_dist.dtype != torch.int64:
        raise ValueError("out_cov and out_dist must be int64 tensors")
    B, M_pad = int(cost.shape[0]), int(cost.shape[1])
    K = int(open_.numel())
    if out_cov.numel() != K * B or out_dist.numel() != K * B:
        raise ValueError("outputs must hold K * B values")
    if base_available is not None and (base_available.dtype != torch.uint8 or base_available.numel() != B):
        raise ValueError("base_available must be a uint8 tensor of B values")
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    err = C.create_string_buffer(512)
    rc = lib().stage_evaluate_swaps_noalloc(
        cost.data_ptr(), B, M, M_pad, None if base_available is None else base_available.data_ptr(),
        open_.data_ptr(), K, R, out_cov.data_ptr(), out_dist.data_ptr(), s, err, 512)
    if rc != STAGE_OK:
        raise StageError(rc, err.value.decode(errors="replace"))


stage_evaluate_swaps_noalloc = evaluate_swaps_noalloc


def batch_schedule(us, gang, P: int):
    """stage_test_batch_schedule (host logic, no device): the placement a
    stage_tabu_batch call uses for searches of estimated times `us` on gangs of
    `gang` CTAs over P CTAs.  Returns (lists, makespan_us): lists[q] = CTA q's
    (search, rank) entries in the order it runs them."""
    us = np.ascontiguousarray(us, dtype=np.float64)
    g = np.ascontiguousarray(gang, dtype=np.int32)
    n = int(us.size)
    if g.size != n:
        raise ValueError("us and gang differ in length")
    off = np.empty(P + 1, dtype=np.int32)
    ent = np.empty(max(1, 2 * int(g.sum()) if n else 1), dtype=np.int32)
    mk = C.c_double()
    rc = lib().stage_test_batch_schedule(n, _ptr(us) if n else None, _ptr(g) if n else None, P, _ptr(off),
                                         _ptr(ent), C.byref(mk))
    if rc != STAGE_OK:
        raise StageError(rc, "stage_test_batch_schedule refused its arguments")
    lists = [[(int(ent[2 * e]), int(ent[2 * e + 1])) for e in range(off[q], off[q + 1])] for q in range(P)]
    return lists, mk.value


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


# C-named entry points (same calls as the Context methods)
def stage_create(**kw) -> Context:
    return Context(**kw)


def stage_destroy(ctx: Context):
    ctx.close()


stage_load_instance = Context.load_instance
stage_unload_instance = Context.unload_instance
stage_rank_bases = Context.rank_bases
stage_evaluate_placement = Context.evaluate_placement
stage_evaluate_swaps = Context.evaluate_swaps
stage_tabu_run = Context.tabu_run
stage_tabu_batch = Context.tabu_batch
stage_local_search = Context.local_search
stage_fleet_tabu = Context.fleet_tabu
stage_best_two = Context.best_two
stage_read_table = Context.read_table
stage_update_instance = Context.update_instance
stage_batch_submit = Context.batch_submit
stage_poll = Context.poll
stage_autotune = Context.autotune
stage_kernel_stats = Context.kernel_stats
stage_reset_stats = Context.reset_stats
