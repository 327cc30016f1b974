"""The seeded input generators: their counter stream matches SplitMix64's
published outputs, and the hypergraphs they build have the stated shape
(source first, distinct sorted targets, sizes in range) and are the same on
every call."""
import numpy as np

from paper_2605_20497_gb300 import inputs


def test_splitmix64_published_values():
    # the first three outputs of SplitMix64 started from state 0 (Steele,
    # Lea, Flood 2014; the reference sequence of its C implementation)
    x = np.array([0, 0x9E3779B97F4A7C15, (2 * 0x9E3779B97F4A7C15) % 2**64], dtype=np.uint64)
    got = [int(v) for v in inputs.splitmix64(x)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def check_shape(g, k_max=None):
    off = g.offsets.astype(np.int64)
    assert off[0] == 0 and (np.diff(off) >= 1).all() and off[-1] == g.pins.size
    for e in range(g.num_hedges):
        seg = g.pins[off[e]:off[e + 1]]
        assert seg[0] == e
        assert (np.diff(seg[1:]) > 0).all() and (seg[1:] != e).all()
        assert seg.min() >= 0 and seg.max() < g.num_nodes
        if k_max:
            assert seg.size <= k_max


def test_random_snn_shape_and_determinism():
    g = inputs.random_snn(600, 31, seed=2)
    check_shape(g)
    assert (np.diff(g.offsets) == 32).all()
    assert np.array_equal(g.pins, inputs.random_snn(600, 31, seed=2).pins)
    assert not np.array_equal(g.pins, inputs.random_snn(600, 31, seed=3).pins)


def test_powerlaw_snn_shape_and_sizes():
    g = inputs.powerlaw_snn(2000, seed=4)
    check_shape(g, k_max=1024)
    sz = np.diff(g.offsets)
    assert sz.min() >= 2 and 4 < sz.mean() < 12          # alpha = 2.2 on [2, 1024]: mean about 7
    assert (sz == 2).mean() > 0.3                          # the mode is the smallest size
    small = inputs.powerlaw_snn(40, seed=1)                # sizes capped by the node count
    check_shape(small, k_max=40)


def test_batch_snn_parameters():
    b = inputs.batch_snn(12, seed=3, n_min=200, n_max=2000)
    assert len(b) == 12
    for g, om, de, sd in b:
        assert 200 <= g.num_nodes <= 2000
        assert om in (256, 512, 1024, 2048, 4096) and de == 4 * om
    again = inputs.batch_snn(12, seed=3, n_min=200, n_max=2000)
    assert all(np.array_equal(a[0].pins, c[0].pins) for a, c in zip(b, again))
