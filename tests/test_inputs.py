"""The seeded input generators: their counter stream matches SplitMix64's
published outputs, and the hypergraphs they build have the stated shape
(source first, distinct sorted targets, sizes in range) and are the same on
every call."""
import numpy as np
import pytest

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


def test_gaussian_offsets_are_centred_binomial():
    e = np.arange(200_000, dtype=np.int64) % 5000
    j = np.arange(200_000, dtype=np.int64) // 5000
    d = inputs.gaussian_offsets(0, 1, e, j)
    assert d.min() >= -32 and d.max() <= 32
    assert abs(d.mean()) < 0.03 and abs(d.var() - 16.0) < 0.2          # B(64, 1/2) - 32: variance 16
    # the exact law: P(d = k) = C(64, 32 + k) / 2^64
    from math import comb
    for k in (0, 3, -6):
        want = comb(64, 32 + k) / 2.0 ** 64
        assert abs(np.mean(d == k) - want) < 5 * np.sqrt(want / d.size)
    dx = inputs.gaussian_offsets(0, 2, e, j)
    assert abs(np.corrcoef(d, dx)[0, 1]) < 0.01                          # the two axes are independent streams


def test_gaussian_layered_snn_structure():
    layers, h, w, mean, cap = 4, 40, 48, 20, 64
    g = inputs.gaussian_layered_snn(layers, h, w, mean, cap, seed=3, chunk=1000)
    n_layer = h * w
    assert g.num_nodes == layers * n_layer and g.num_hedges == (layers - 1) * n_layer
    off = g.offsets.astype(np.int64)
    sizes = np.diff(off)
    assert sizes.min() >= 1 and sizes.max() <= cap
    for e in range(0, g.num_hedges, 37):
        row = g.pins[off[e]:off[e + 1]].astype(np.int64)
        assert row[0] == e                                               # the source first
        t = row[1:]
        assert np.all(np.diff(t) > 0)                                    # distinct, ascending
        assert np.all(t // n_layer == e // n_layer + 1)                  # all in the next layer
        dy = (t % n_layer) // w - (e % n_layer) // w
        dx = t % w - e % w
        assert np.all(np.abs(dy) <= 32) and np.all(np.abs(dx) <= 32)
    # away from the border, sizes follow min(geometric(mean), cap): E = mean (1 - (1 - 1/mean)^cap)
    e = np.arange(g.num_hedges)
    y, x = (e % n_layer) // w, e % w
    inner = (y >= 12) & (y < h - 12) & (x >= 12) & (x < w - 12)
    want = mean * (1 - (1 - 1 / mean) ** cap)
    assert abs(sizes[inner].mean() - want) < 0.06 * want


def test_gaussian_layered_snn_deterministic_and_chunk_independent():
    a = inputs.gaussian_layered_snn(3, 24, 24, 16, 64, seed=1, chunk=100)
    b = inputs.gaussian_layered_snn(3, 24, 24, 16, 64, seed=1, chunk=1 << 16)
    c = inputs.gaussian_layered_snn(3, 24, 24, 16, 64, seed=1, chunk=150, workers=2)
    d = inputs.gaussian_layered_snn(3, 24, 24, 16, 64, seed=2)
    for x in (b, c):
        assert np.array_equal(a.offsets, x.offsets) and np.array_equal(a.pins, x.pins)
    assert not np.array_equal(a.pins, d.pins)


def test_geometric_thresholds_exact():
    t = inputs._geometric_thresholds(84, 1024)
    assert t.size == 1023 and np.all(np.diff(t) > 0)
    assert t[-1] == 83 / 84 and t[0] == pytest.approx((83 / 84) ** 1023, rel=1e-12)
