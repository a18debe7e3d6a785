"""Seeded synthetic staging instances (bases, facilities, missions).

This module only draws coordinates and sizes.  It holds none of the method's
arithmetic (no legs, costs, rankings or objectives), so both the CUDA path and
the CPU oracle can be fed from it without sharing any of the method.

Shapes follow the paper's workloads (Sec. 3 and Sec. 5: candidate bases, health
facilities, missions that go base -> pickup -> facility drop-off -> same base),
scaled up: integer-metre planar coordinates (Sec. 3 allows a Euclidean metric for
simulated data), a uniform box or 80 % of the points in 6 Gaussian clusters
inside the southern 20 % strip of the box with the other 20 % uniform over the
rest of the box, resampling Gaussian points that fall outside the box.

Random numbers come from SplitMix64 (Steele, Lea and Flood, 2014) used as a
counter-based generator: the k-th output of the stream with key s is
``mix64(s + (k + 1) * 0x9E3779B97F4A7C15)``, which is exactly the k-th output of a
SplitMix64 generator seeded with s.  Each entity class (bases, facilities,
pickups, drop-off choice, sizes, arrivals) and each resampling attempt has its
own key, so every draw can be computed independently and vectorised.  Gaussians
use the Box-Muller transform in float64; coordinates are rounded to whole metres.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

# entity classes (stream identifiers)
CLS_BASES, CLS_FACILITIES, CLS_PICKUPS, CLS_DROPOFF, CLS_SIZES, CLS_ARRIVALS, CLS_UPDATES = 1, 2, 3, 4, 5, 6, 7
CLS_SCAN = 8   # scan orders of the local search
CLS_TYPES = 9  # base and mission types of the heterogeneous fleet

# Draws consumed per point and attempt: [mixture choice, cluster id, u1, u2].
_DRAWS_PER_POINT = 4
_MAX_ATTEMPTS = 64


def _mix64_int(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(_M1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(_M2)
    z ^= z >> np.uint64(31)
    return z


def scan_orders(seed: int, n_passes: int, K: int, nC: int):
    """The local search's random scan orders (Alg. 2 draws two permutations per
    pass): pass p's slot order and candidate-position order, each the stable
    argsort of fresh SplitMix64 draws.  Returns int32 arrays [n_passes, K] and
    [n_passes, nC]."""
    ps = np.empty((n_passes, K), dtype=np.int32)
    pc = np.empty((n_passes, nC), dtype=np.int32)
    for p in range(n_passes):
        ks = draws_u64(stream_key(seed, CLS_SCAN, 2 * p), np.arange(K))
        kc = draws_u64(stream_key(seed, CLS_SCAN, 2 * p + 1), np.arange(nC))
        ps[p] = np.argsort(ks, kind="stable")
        pc[p] = np.argsort(kc, kind="stable")
    return ps, pc


def stream_key(seed: int, cls: int, sub: int = 0) -> int:
    """Key of the SplitMix64 stream for (seed, entity class, sub-stream)."""
    k = _mix64_int(seed * GOLDEN_GAMMA + 0x632BE59BD9B4E019)
    k = _mix64_int(k ^ ((cls * 0xD1342543DE82EF95) & _MASK))
    return _mix64_int(k ^ ((sub * 0xA0761D6478BD642F + 1) & _MASK))


def draws_u64(key: int, counters: np.ndarray) -> np.ndarray:
    """Outputs number ``counters`` (0-based) of the SplitMix64 stream ``key``."""
    c = np.asarray(counters, dtype=np.uint64)
    return _mix64(np.uint64(key) + (c + np.uint64(1)) * np.uint64(GOLDEN_GAMMA))


def u01(u: np.ndarray) -> np.ndarray:
    """Top 53 bits of a uint64 as a float64 in [0, 1)."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Layout:
    """Spatial distribution of points: a box in metres, optional clusters."""
    width_m: int
    height_m: int
    clustered: bool = False
    n_clusters: int = 6
    sigma_m: float = 0.0
    cluster_frac: float = 0.8
    strip_frac: float = 0.2


def _cluster_centres(seed: int, lay: Layout) -> np.ndarray:
    key = stream_key(seed, 0, 0xC)
    u = u01(draws_u64(key, np.arange(2 * lay.n_clusters)))
    cx = np.floor(u[0::2] * lay.width_m)
    cy = np.floor(u[1::2] * (lay.strip_frac * lay.height_m))
    return np.stack([cx, cy], axis=1)


def draw_points(seed: int, cls: int, n: int, lay: Layout, centres: np.ndarray | None) -> np.ndarray:
    """n int32 (x, y) points from the layout; Gaussian points outside the box are redrawn."""
    out = np.zeros((n, 2), dtype=np.int64)
    todo = np.arange(n, dtype=np.int64)
    W, H = lay.width_m, lay.height_m
    strip = int(math.floor(lay.strip_frac * H))
    for attempt in range(_MAX_ATTEMPTS):
        if todo.size == 0:
            break
        key = stream_key(seed, cls, attempt)
        base = todo.astype(np.uint64) * np.uint64(_DRAWS_PER_POINT)
        d = [u01(draws_u64(key, base + np.uint64(k))) for k in range(_DRAWS_PER_POINT)]
        if not lay.clustered:
            x = np.floor(d[2] * W)
            y = np.floor(d[3] * H)
            out[todo, 0] = x.astype(np.int64)
            out[todo, 1] = y.astype(np.int64)
            todo = todo[:0]
            break
        in_cluster = d[0] < lay.cluster_frac
        # uniform part: the box outside the southern strip
        ux = np.floor(d[2] * W)
        uy = strip + np.floor(d[3] * (H - strip))
        # clustered part: Box-Muller around a centre
        cid = np.minimum(np.floor(d[1] * lay.n_clusters).astype(np.int64), lay.n_clusters - 1)
        r = np.sqrt(-2.0 * np.log1p(-d[2]))
        g1 = r * np.cos(2.0 * np.pi * d[3])
        g2 = r * np.sin(2.0 * np.pi * d[3])
        gx = np.rint(centres[cid, 0] + lay.sigma_m * g1)
        gy = np.rint(centres[cid, 1] + lay.sigma_m * g2)
        x = np.where(in_cluster, gx, ux)
        y = np.where(in_cluster, gy, uy)
        ok = (x >= 0) & (x < W) & (y >= 0) & (y < H)
        done = todo[ok]
        out[done, 0] = x[ok].astype(np.int64)
        out[done, 1] = y[ok].astype(np.int64)
        todo = todo[~ok]
    if todo.size:
        raise RuntimeError("point resampling did not converge")
    return out.astype(np.int32)


@dataclass
class Instance:
    """One staging instance: B candidate bases, M missions, K vehicles, range R (metres)."""
    name: str
    seed: int
    base_xy: np.ndarray      # int32 [B, 2]
    pick_xy: np.ndarray      # int32 [M, 2]
    drop_xy: np.ndarray      # int32 [M, 2]
    K: int
    R: int
    iters: int
    tenure: int
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.base_xy.shape[0])

    @property
    def M(self) -> int:
        return int(self.pick_xy.shape[0])

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.base_xy, self.pick_xy, self.drop_xy):
            h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
        h.update(np.array([self.K, self.R, self.iters, self.tenure], dtype=np.int64).tobytes())
        return h.hexdigest()[:16]


def make_instance(name: str, seed: int, B: int, n_facilities: int, M: int, K: int, R: int,
                  iters: int, tenure: int, lay: Layout) -> Instance:
    centres = _cluster_centres(seed, lay) if lay.clustered else None
    bases = draw_points(seed, CLS_BASES, B, lay, centres)
    facs = draw_points(seed, CLS_FACILITIES, n_facilities, lay, centres)
    picks = draw_points(seed, CLS_PICKUPS, M, lay, centres)
    key = stream_key(seed, CLS_DROPOFF, 0)
    choice = np.floor(u01(draws_u64(key, np.arange(M))) * n_facilities).astype(np.int64)
    choice = np.minimum(choice, n_facilities - 1)
    drops = facs[choice]
    meta = dict(width_m=lay.width_m, height_m=lay.height_m, clustered=lay.clustered,
                sigma_m=lay.sigma_m, n_facilities=n_facilities)
    return Instance(name, seed, bases, picks, np.ascontiguousarray(drops), K, R, iters, tenure, meta)


KM = 1000


def tiny(seed: int = 0) -> Instance:
    """B=20, 40 facilities, M=200, uniform 1000x1000 km, K=5, R=800 km, 100 it, tenure 7."""
    lay = Layout(1000 * KM, 1000 * KM)
    return make_instance("tiny", seed, 20, 40, 200, 5, 800 * KM, 100, 7, lay)


def province(seed: int = 1) -> Instance:
    """B=300, 600 facilities, M=20,000, clustered 1500x1700 km (sigma 60 km), K=12, R=1000 km."""
    lay = Layout(1500 * KM, 1700 * KM, clustered=True, sigma_m=60.0 * KM)
    return make_instance("province", seed, 300, 600, 20000, 12, 1000 * KM, 500, 15, lay)


def large(seed: int = 2, M: int = 1_000_000, B: int = 2000) -> Instance:
    """B=2000, 4000 facilities, M=1e6, clustered 3000x3000 km (sigma 120 km), K=64, R=1200 km."""
    lay = Layout(3000 * KM, 3000 * KM, clustered=True, sigma_m=120.0 * KM)
    return make_instance("large", seed, B, 2 * B, M, 64, 1200 * KM, 1000, 25, lay)


# Geographic instances (Eq. 1 legs): (latitude, longitude) in microdegrees over
# a 15 x 21 degree region with its clusters in the southern strip (the layout of
# the province workload, drawn on a latitude / longitude box).
GEO_LAT0, GEO_LON0 = 42_000_000, -95_000_000
GEO_LAT_SPAN, GEO_LON_SPAN = 15_000_000, 21_000_000


def geo_instance(name: str, seed: int, B: int, M: int, K: int, R: int, iters: int, tenure: int,
                 n_facilities: int | None = None) -> Instance:
    """An instance whose coordinates are (latitude, longitude) microdegree pairs."""
    lay = Layout(GEO_LON_SPAN, GEO_LAT_SPAN, clustered=True, sigma_m=300_000.0)
    inst = make_instance(name, seed, B, n_facilities or 2 * B, M, K, R, iters, tenure, lay)

    def to_geo(xy):
        out = np.empty_like(xy)
        out[:, 0] = GEO_LAT0 + xy[:, 1]   # the layout's y (strip = south) is latitude
        out[:, 1] = GEO_LON0 + xy[:, 0]
        return out.astype(np.int32)

    inst.base_xy, inst.pick_xy, inst.drop_xy = to_geo(inst.base_xy), to_geo(inst.pick_xy), to_geo(inst.drop_xy)
    inst.meta = dict(inst.meta, coordinates="latitude, longitude (microdegrees)")
    return inst


def geo_paper(seed: int = 5) -> Instance:
    """The paper's own scale on Eq. 1 legs: B=378 bases, M=180 missions, K=12; R=1500 km, 200 it, tenure 7."""
    return geo_instance("geo_paper", seed, 378, 180, 12, 1500 * KM, 200, 7)


def fleet_types(seed: int, B: int, M: int, n_helipads: int, rotary_frac: float):
    """Base and mission types of a heterogeneous fleet: n_helipads of the B bases
    are helipads (the rest aerodromes) and about rotary_frac of the missions
    need a rotary-wing vehicle; returns uint8 arrays [B], [M]."""
    kb = draws_u64(stream_key(seed, CLS_TYPES, 0), np.arange(B))
    heli = np.zeros(B, dtype=np.uint8)
    heli[np.argsort(kb, kind="stable")[:n_helipads]] = 1
    rot = (u01(draws_u64(stream_key(seed, CLS_TYPES, 1), np.arange(M))) < rotary_frac).astype(np.uint8)
    return heli, rot


def fleet_paper(seed: int = 5):
    """The paper's fleet (Sec. 5): 378 bases of which 104 helipads, 8 rotary-wing
    and 4 fixed-wing vehicles, 180 missions (30 % rotary-only), Eq. 1 legs.
    Returns (instance, helipad mask, rotary-only mask, K_rotary, K_fixed)."""
    inst = geo_paper(seed)
    heli, rot = fleet_types(seed, inst.B, inst.M, 104, 0.3)
    return inst, heli, rot, 8, 4


def batched_sizes(seed: int = 3, n: int = 512):
    """Per-instance (B, M, K, R) of the batched workload, drawn log-uniform / uniform."""
    key = stream_key(seed, CLS_SIZES, 0)
    u = u01(draws_u64(key, np.arange(4 * n))).reshape(n, 4)
    B = np.rint(np.exp(math.log(50) + u[:, 0] * (math.log(800) - math.log(50)))).astype(np.int64)
    M = np.rint(np.exp(math.log(1e3) + u[:, 1] * (math.log(2e5) - math.log(1e3)))).astype(np.int64)
    K = 4 + np.minimum(np.floor(u[:, 2] * 29), 28).astype(np.int64)
    R = np.rint((600.0 + u[:, 3] * 600.0) * KM).astype(np.int64)
    K = np.minimum(K, B - 1)
    return [(int(B[i]), int(M[i]), int(K[i]), int(R[i])) for i in range(n)]


def batched_instance(seed: int, index: int, B: int, M: int, K: int, R: int,
                     iters: int = 300, tenure: int = 11) -> Instance:
    lay = Layout(1500 * KM, 1700 * KM, clustered=True, sigma_m=60.0 * KM)
    sub_seed = _mix64_int(seed * GOLDEN_GAMMA + index + 1) & 0x7FFFFFFFFFFFFFFF
    return make_instance(f"batched[{index}]", sub_seed, B, 2 * B, M, K, R, iters, tenure, lay)


def batched(seed: int = 3, n: int = 512, scale_m: float = 1.0):
    """The batched workload: n independent instances of uneven B, M, K, R."""
    out = []
    for i, (B, M, K, R) in enumerate(batched_sizes(seed, n)):
        out.append(batched_instance(seed, i, B, max(1, int(round(M * scale_m))), K, R))
    return out


def by_name(name: str) -> Instance:
    return {"tiny": tiny, "province": province, "large": large, "geo": geo_paper}[name]()
