"""The seeded input generator: SplitMix64 stream and workload shapes."""
import numpy as np

from paper_1811_03882_gb300 import synth


def _splitmix_py(seed, i):
    """SplitMix64 written out with Python integers (draw i, 0-based)."""
    M = (1 << 64) - 1
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix_matches_integer_definition():
    for seed in (0, 1, 101, (4 << 32) + 7):
        got = synth.splitmix64(seed, 5, 20)
        ref = [_splitmix_py(seed, i) for i in range(5, 25)]
        assert [int(v) for v in got] == ref


def test_stream_is_sequential():
    a = synth.Stream(3)
    u1, u2 = a.uniform(10), a.uniform(7)
    b = synth.Stream(3).uniform(17)
    np.testing.assert_array_equal(np.concatenate([u1, u2]), b)


def test_distributions():
    s = synth.Stream(9)
    u = s.uniform(200000, -1, 1)
    assert -1 <= u.min() and u.max() < 1 and abs(u.mean()) < 0.01
    n = s.normal(200000, 2.0)
    assert abs(n.mean()) < 0.02 and abs(n.std() - 2.0) < 0.02


def test_network_shapes_and_flops():
    n9, n19 = synth.net_9conv(), synth.net_19conv()
    assert len(n9.layers) == 9 and len(n19.layers) == 19
    assert n9.out_hw(416, 416) == (13, 13) and n9.out_c() == 125
    assert n19.out_hw(448, 448) == (14, 14) and n19.out_c() == 1000
    assert abs(n9.conv_flops(1, 416, 416) / 1e9 - 6.971) < 0.01
    assert abs(n19.conv_flops(8, 448, 448) / 1e9 - 178.62) < 0.05
    assert sum(1 for l in n19.layers if l.pool == synth.POOL_2X2S2) == 5


def test_blob_roundtrip():
    spec, x, blob = synth.workload_single()
    assert x.shape == (1, 16, 32, 32) and x.dtype == np.float32
    assert blob.size == spec.n_params()
    ps = synth.unpack_blob(spec, blob)
    np.testing.assert_array_equal(synth.pack_blob(spec, ps), blob)
    p = ps[0]
    assert 0.5 <= p.gamma.min() and p.gamma.max() <= 1.5 and 0.5 <= p.var.min()


def test_uneven_and_arrivals():
    sides = synth.uneven_sides()
    assert sides.size == 64 and set(sides.tolist()) <= {320, 416, 512, 608}
    t, cam, side = synth.poisson_arrivals(1000.0, 2.0)
    assert np.all(np.diff(t) >= 0) and 1700 < t.size < 2300
    assert set(side.tolist()) <= {320, 416, 608} and cam.max() < 32
