"""The seeded input generator: determinism, the published SplitMix64 outputs,
and the shape of the synthetic workloads."""
import numpy as np

from paper_2001_05291_gb300 import synth


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 1234567 (the reference implementation's test vector)
    got = [int(x) for x in synth.draws_u64(1234567, np.arange(3))]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_counter_form_equals_sequential_generator():
    mask = (1 << 64) - 1
    state, out = 987654321, []
    for _ in range(50):
        state = (state + synth.GOLDEN_GAMMA) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    assert [int(x) for x in synth.draws_u64(987654321, np.arange(50))] == out


def test_deterministic_and_seed_dependent():
    assert synth.tiny().digest() == synth.tiny().digest()
    assert synth.tiny(0).digest() != synth.tiny(5).digest()
    a, b = synth.province(), synth.province()
    assert np.array_equal(a.pick_xy, b.pick_xy) and np.array_equal(a.drop_xy, b.drop_xy)


def test_tiny_shape_and_box():
    i = synth.tiny()
    assert (i.B, i.M, i.K, i.R, i.iters, i.tenure) == (20, 200, 5, 800_000, 100, 7)
    for a in (i.base_xy, i.pick_xy, i.drop_xy):
        assert a.dtype == np.int32
        assert a.min() >= 0 and a.max() < 1_000_000
    # drop-offs are facilities: at most 40 distinct points
    assert len({tuple(p) for p in i.drop_xy.tolist()}) <= 40


def test_province_clusters_in_southern_strip():
    i = synth.province()
    assert (i.B, i.M, i.K, i.R) == (300, 20000, 12, 1_000_000)
    W, H = 1_500_000, 1_700_000
    p = i.pick_xy
    assert p[:, 0].min() >= 0 and p[:, 0].max() < W and p[:, 1].min() >= 0 and p[:, 1].max() < H
    # about 80 % of points are clustered near the southern strip (y < 0.2 H + 4 sigma)
    near_south = np.mean(p[:, 1] < 0.2 * H + 4 * 60_000)
    assert 0.75 < near_south < 0.9
    assert len({tuple(q) for q in i.drop_xy.tolist()}) <= 600


def test_batched_size_distribution():
    s = np.array(synth.batched_sizes())
    assert s.shape == (512, 4)
    B, M, K, R = s.T
    assert B.min() >= 50 and B.max() <= 800
    assert M.min() >= 1000 and M.max() <= 200_000
    assert K.min() >= 4 and K.max() <= 32 and np.all(K < B)
    assert R.min() >= 600_000 and R.max() <= 1_200_000
    # log-uniform: the median of B is near sqrt(50 * 800) = 200
    assert 150 < np.median(B) < 260
