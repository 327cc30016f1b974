"""hp_partition_batch: many independent hypergraphs (power-law hyperedge
sizes, uneven node counts, mixed Omega/Delta) in one call.  Every instance
must come out exactly as a single hp_partition call gives it (and as the
oracle gives it), whatever the concurrency, and a failing instance must not
disturb the others."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import hp, inputs

pytestmark = pytest.mark.gpu

STAT_KEYS = ("connectivity", "cut_net", "num_parts", "max_part_size", "max_part_distinct", "violations", "levels",
             "moves_applied")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_20497_gb300 import build
    build.build()
    oracle.build()
    hp.load()
    return t


@pytest.fixture(scope="module")
def graphs():
    return inputs.batch_snn(10, seed=5, n_min=300, n_max=3000)


def same(a, b):
    assert a.status == b.status
    assert np.array_equal(a.part, b.part)
    for k in STAT_KEYS:
        assert a.stats[k] == b.stats[k], k


def test_batch_matches_single_calls_and_oracle(torch, graphs):
    rc, res = hp.partition_batch(graphs, concurrency=4)
    assert rc == hp.HP_OK, hp.hp_last_error()
    for (g, om, de, sd), r in zip(graphs, res):
        assert r.status == hp.HP_OK
        same(r, hp.partition(g, om, de, seed=sd))
    for (g, om, de, sd), r in list(zip(graphs, res))[:3]:
        o = oracle.partition(g, om, de, seed=sd)
        assert o.status == oracle.OK
        assert np.array_equal(r.part, o.part)
        assert r.stats["connectivity"] == o.stats["connectivity"]


def test_batch_independent_of_concurrency(torch, graphs):
    rc1, a = hp.partition_batch(graphs, concurrency=1)
    rc8, b = hp.partition_batch(graphs, concurrency=8)
    assert rc1 == rc8 == hp.HP_OK
    for x, y in zip(a, b):
        same(x, y)


def test_batch_failure_stays_with_its_instance(torch, graphs):
    g0, om, de, sd = graphs[2]
    bad = inputs.Hypergraph(num_nodes=g0.num_nodes, offsets=g0.offsets.copy(), pins=g0.pins.copy())
    bad.pins[5] = g0.num_nodes   # out of range
    mixed = list(graphs[:4])
    mixed[2] = (bad, om, de, sd)
    rc, res = hp.partition_batch(mixed, concurrency=3)
    assert rc == hp.HP_ERR_BAD_CSR
    assert "instance 2" in hp.hp_last_error()
    for i, ((g, om, de, sd), r) in enumerate(zip(mixed, res)):
        if i == 2:
            assert r.status == hp.HP_ERR_BAD_CSR
        else:
            same(r, hp.partition(g, om, de, seed=sd))


def test_batch_arguments(torch):
    lib = hp.load()
    assert lib.hp_partition_batch(None, 0, None, 4, None, None, None) == hp.HP_OK
    assert lib.hp_partition_batch(None, 1, None, 4, None, None, None) == hp.HP_ERR_INVALID_ARG
    one = (hp.hp_instance * 1)()
    assert lib.hp_partition_batch(one, 1, None, 0, None, None, None) == hp.HP_ERR_INVALID_ARG
    assert ctypes.sizeof(hp.hp_instance) == 64


def test_autotuned_batch_matches_single_calls(torch):
    """concurrency 0: the size-class autotuner only changes the schedule;
    every instance is the single call's, bit for bit, and the classes with
    enough instances get a tuned concurrency."""
    graphs = inputs.batch_snn(40, seed=6, n_min=500, n_max=6000)
    rc, res = hp.partition_batch(graphs, concurrency=0)
    assert rc == hp.HP_OK, hp.hp_last_error()
    for (g, om, de, sd), r in zip(graphs, res):
        same(r, hp.partition(g, om, de, seed=sd))
    dev = torch.cuda.current_device()
    lib = hp.load()
    tuned = [lib.hp_batch_tuned_concurrency(dev, c) for c in range(6)]
    assert all(t in (0, 4, 8, 16, 32, 64) for t in tuned)
    # a second call with the same classes reuses the tuned schedule
    rc2, res2 = hp.partition_batch(graphs, concurrency=0)
    assert rc2 == hp.HP_OK
    for a, b in zip(res, res2):
        same(a, b)
