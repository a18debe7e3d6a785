"""Pins of the oracle's Haversine legs (Eq. 1) on (latitude, longitude) microdegrees.

* closed forms: along the equator and along a meridian the great-circle
  distance is r times the angle; antipodal points are pi r apart;
* an independent formula: the arctangent form of the great-circle distance,
  written here in Python doubles, agrees to within a micrometre before the
  rounding up, so the rounded legs agree wherever the distance is not within a
  micrometre of a whole metre;
* symmetry and the table as the sum of the mission's three legs.
"""
import math

import numpy as np

from paper_2001_05291_gb300 import synth

R_EARTH = 6371000.0
RAD = math.pi / 180.0 * 1e-6


def ceil_if_clear(d: float):
    """ceil(d), or None when d is within a micrometre of a whole metre."""
    if abs(d - round(d)) < 1e-6:
        return None
    return math.ceil(d)


def great_circle(lat1, lon1, lat2, lon2):
    p1, p2, dl = lat1 * RAD, lat2 * RAD, (lon2 - lon1) * RAD
    y = math.hypot(math.cos(p2) * math.sin(dl), math.cos(p1) * math.sin(p2) - math.sin(p1) * math.cos(p2) * math.cos(dl))
    x = math.sin(p1) * math.sin(p2) + math.cos(p1) * math.cos(p2) * math.cos(dl)
    return R_EARTH * math.atan2(y, x)


def test_equator_meridian_and_antipodes(orc):
    checked = 0
    for deg_u in (1, 999, 1_000_000, 12_345_678, 90_000_000, 179_999_999):
        for want_d, got in ((R_EARTH * deg_u * RAD, orc.leg_haversine(0, 0, 0, deg_u)),
                            (R_EARTH * deg_u * RAD if deg_u <= 90_000_000 else None,
                             orc.leg_haversine(0, 0, min(deg_u, 90_000_000), 0))):
            if want_d is None:
                continue
            want = ceil_if_clear(want_d)
            if want is not None:
                assert got == want
                checked += 1
    assert checked >= 8
    assert orc.leg_haversine(0, 0, 0, 180_000_000) == math.ceil(math.pi * R_EARTH)
    assert orc.leg_haversine(45_000_000, 10_000_000, -45_000_000, -170_000_000) == math.ceil(math.pi * R_EARTH)
    assert orc.leg_haversine(45_000_000, -75_000_000, 45_000_000, -75_000_000) == 0


def test_agrees_with_the_arctangent_form_and_is_symmetric(orc):
    key = synth.stream_key(77, 91, 0)
    u = synth.u01(synth.draws_u64(key, np.arange(4 * 4000))).reshape(-1, 4)
    lat = np.floor((u[:, 0] * 2 - 1) * 89_000_000).astype(np.int64)
    lon = np.floor((u[:, 1] * 2 - 1) * 180_000_000).astype(np.int64)
    lat2 = np.floor((u[:, 2] * 2 - 1) * 89_000_000).astype(np.int64)
    lon2 = np.floor((u[:, 3] * 2 - 1) * 180_000_000).astype(np.int64)
    n = 0
    for a, b, c, d in zip(lat, lon, lat2, lon2):
        got = orc.leg_haversine(int(a), int(b), int(c), int(d))
        assert got == orc.leg_haversine(int(c), int(d), int(a), int(b))
        want = ceil_if_clear(great_circle(int(a), int(b), int(c), int(d)))
        if want is not None:
            assert got == want, (a, b, c, d)
            n += 1
    assert n > 3900


def test_geo_table_is_the_sum_of_three_legs(orc):
    inst = synth.geo_instance("g", 3, 12, 40, 3, 900_000, 10, 3)
    cost = orc.cost_table(inst.base_xy, inst.pick_xy, inst.drop_xy, 2, haversine=True)
    for b in range(inst.B):
        for m in range(0, inst.M, 7):
            (bl, bo), (pl, po), (dl, do) = inst.base_xy[b], inst.pick_xy[m], inst.drop_xy[m]
            want = (orc.leg_haversine(int(bl), int(bo), int(pl), int(po)) +
                    orc.leg_haversine(int(pl), int(po), int(dl), int(do)) +
                    orc.leg_haversine(int(dl), int(do), int(bl), int(bo)))
            assert cost[b, m] == want
    # a degree of latitude is about 111 km: the table is in metres on the sphere
    assert 10_000 < int(np.median(cost)) < 5_000_000


def test_geo_generator_ranges():
    inst = synth.geo_paper()
    for xy in (inst.base_xy, inst.pick_xy, inst.drop_xy):
        assert (xy[:, 0] >= synth.GEO_LAT0).all() and (xy[:, 0] <= synth.GEO_LAT0 + synth.GEO_LAT_SPAN).all()
        assert (xy[:, 1] >= synth.GEO_LON0).all() and (xy[:, 1] <= synth.GEO_LON0 + synth.GEO_LON_SPAN).all()
    assert (inst.B, inst.M, inst.K) == (378, 180, 12)
