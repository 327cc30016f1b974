"""hp_connectivity_noalloc (the entry point that uses only the library's
fixed scratch area) against hp_connectivity and the oracle, on hyperedges of
every size class (one warp, one CTA in shared memory, one CTA on a region of
the scratch table), two calls in a row, and after a rejected call.  Named to
run last so that it also runs after everything else has used the device."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import hp, inputs

pytestmark = pytest.mark.gpu

LIMIT = 262_144


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


def mixed_graph(seed, sizes, n):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n, size=s, replace=False)).astype(np.int32) for s in sizes]
    offsets = np.zeros(len(rows) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum([len(r) for r in rows])
    pins = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    w = rng.integers(1, 65537, len(rows)).astype(np.int32)
    return inputs.Hypergraph(num_nodes=n, offsets=offsets, pins=pins, weights=w, name=f"mixed_{seed}")


def sizes_of(seed):
    rng = np.random.default_rng(seed)
    small = list(rng.integers(1, 257, 3000))
    mid = list(rng.integers(257, 8193, 40))
    large = [8193, 50_000, LIMIT]
    out = small + mid + large
    rng.shuffle(out)
    return [int(s) for s in out]


def call(fn, torch, g, rho, nparts, weights=True):
    d = hp.to_device(g)
    part = torch.from_numpy(rho).cuda()
    w = d["weights"].data_ptr() if weights else None
    return fn(d["pins"].data_ptr(), d["offsets"].data_ptr(), g.num_hedges, w, part.data_ptr(), g.num_nodes, nparts)


@pytest.mark.parametrize("seed", [0, 1])
def test_noalloc_equals_existing_entry_point_twice(torch, seed):
    n = 300_000
    g = mixed_graph(seed, sizes_of(seed), n)
    nparts = 97
    rho = np.random.default_rng(seed + 10).integers(0, nparts, n).astype(np.int32)
    first = call(hp.hp_connectivity_noalloc, torch, g, rho, nparts)
    second = call(hp.hp_connectivity_noalloc, torch, g, rho, nparts)
    ref = call(hp.hp_connectivity, torch, g, rho, nparts)
    assert first[0] == hp.HP_OK, hp.hp_last_error()
    assert first == second == ref
    assert first[1:] == oracle.objective(g, rho, nparts)
    # unit weights (NULL) as well
    a = call(hp.hp_connectivity_noalloc, torch, g, rho, nparts, weights=False)
    b = call(hp.hp_connectivity, torch, g, rho, nparts, weights=False)
    assert a == b and a[0] == hp.HP_OK


def test_noalloc_few_parts_and_layered(torch):
    g = inputs.workload("layered_snn_16k")
    for nparts, seed in ((1, 0), (2, 1), (5000, 2)):
        rho = np.random.default_rng(seed).integers(0, nparts, g.num_nodes).astype(np.int32)
        a = call(hp.hp_connectivity_noalloc, torch, g, rho, nparts, weights=False)
        b = call(hp.hp_connectivity, torch, g, rho, nparts, weights=False)
        assert a == b and a[0] == hp.HP_OK


def test_noalloc_rejects_oversize_and_stays_clean(torch):
    n = 300_000
    g = mixed_graph(5, [10, 300, LIMIT + 1, 9000], n)
    rho = np.random.default_rng(6).integers(0, 11, n).astype(np.int32)
    st, _, _ = call(hp.hp_connectivity_noalloc, torch, g, rho, 11)
    assert st == hp.HP_ERR_INVALID_ARG
    assert str(LIMIT + 1) in hp.hp_last_error() and str(LIMIT) in hp.hp_last_error()
    ok = mixed_graph(7, sizes_of(7), n)
    a = call(hp.hp_connectivity_noalloc, torch, ok, rho, 11)
    b = call(hp.hp_connectivity, torch, ok, rho, 11)
    assert a == b and a[0] == hp.HP_OK


def test_noalloc_errors_and_empty(torch):
    g = inputs.random_hypergraph(200, 300, 12, seed=4, weights=True)
    rho = np.random.default_rng(0).integers(0, 5, 200).astype(np.int32)
    assert call(hp.hp_connectivity_noalloc, torch, g, rho, 4)[0] == hp.HP_ERR_INVALID_ARG  # part id 4 >= 4
    bad = inputs.Hypergraph(num_nodes=200, offsets=g.offsets.copy(), pins=g.pins.copy(), weights=g.weights)
    bad.pins[3] = 200
    assert call(hp.hp_connectivity_noalloc, torch, bad, rho, 5)[0] == hp.HP_ERR_BAD_CSR
    bad2 = inputs.Hypergraph(num_nodes=200, offsets=g.offsets.copy(), pins=g.pins, weights=g.weights)
    bad2.offsets[5] = bad2.offsets[4]
    assert call(hp.hp_connectivity_noalloc, torch, bad2, rho, 5)[0] == hp.HP_ERR_BAD_CSR
    assert call(hp.hp_connectivity_noalloc, torch, g, rho, 5) == call(hp.hp_connectivity, torch, g, rho, 5)
    empty = inputs.Hypergraph(num_nodes=3, offsets=np.zeros(1, np.int32), pins=np.zeros(0, np.int32))
    z = call(hp.hp_connectivity_noalloc, torch, empty, np.zeros(3, np.int32), 1, weights=False)
    assert z == (hp.HP_OK, 0, 0)
    st = hp.load().hp_connectivity_noalloc(None, None, -1, None, None, 0, 0, None, None, None)
    assert st == hp.HP_ERR_INVALID_ARG


ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def test_noalloc_works_while_the_allocator_refuses(torch):
    """With an allocator hook that refuses every request, hp_connectivity
    fails for lack of workspace while hp_connectivity_noalloc still returns
    the same numbers; and a call after a first call takes no device memory."""
    n = 300_000
    g = mixed_graph(11, sizes_of(11), n)
    rho = np.random.default_rng(12).integers(0, 31, n).astype(np.int32)
    ref = call(hp.hp_connectivity, torch, g, rho, 31)
    assert ref[0] == hp.HP_OK
    d = hp.to_device(g)
    part = torch.from_numpy(rho).cuda()
    args = (d["pins"].data_ptr(), d["offsets"].data_ptr(), g.num_hedges, d["weights"].data_ptr(), part.data_ptr(),
            n, 31)
    assert hp.hp_connectivity_noalloc(*args) == ref          # first call on this device done
    torch.cuda.synchronize()
    requests = []
    refuse = ALLOC_T(lambda size, ctx: requests.append(size))   # returns None: refused
    never = FREE_T(lambda p, ctx: None)
    L = hp.load()
    assert L.hp_set_allocator(ctypes.cast(refuse, ctypes.c_void_p), ctypes.cast(never, ctypes.c_void_p), None) == 0
    try:
        free0 = torch.cuda.mem_get_info()[0]
        a = hp.hp_connectivity_noalloc(*args)
        b = hp.hp_connectivity_noalloc(*args)
        free1 = torch.cuda.mem_get_info()[0]
        assert requests == []
        assert a == b == ref
        assert free1 == free0
        st = hp.hp_connectivity(*args)[0]
        assert st == hp.HP_ERR_OOM and len(requests) >= 1
    finally:
        assert L.hp_set_allocator(None, None, None) == 0
    assert call(hp.hp_connectivity, torch, g, rho, 31) == ref
