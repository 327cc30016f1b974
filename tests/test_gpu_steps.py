"""GPU step parity: one coarsening level and one refinement repetition
through the step-level ABI entry points, against the oracle's steps."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import hp, inputs

pytestmark = pytest.mark.gpu


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


def dev(torch, a, dtype=None):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a).cuda()


def level_arrays(torch, g, size):
    src = g.src_counts if g.src_counts is not None else np.ones(g.num_hedges, np.int32)
    w = g.weights if g.weights is not None else np.ones(g.num_hedges, np.int32)
    pins = g.pins if g.num_pins else np.zeros(1, np.int32)
    return dict(off=dev(torch, g.offsets.astype(np.int32)), pins=dev(torch, pins.astype(np.int32)),
                src=dev(torch, np.asarray(src, np.int32)), w=dev(torch, np.asarray(w, np.int32)),
                size=dev(torch, np.asarray(size, np.int32)))


def gpu_coarsen(torch, g, size, omega, delta, seed, level, **opts):
    d = level_arrays(torch, g, size)
    o = hp.options(**opts)
    n, pi = g.num_nodes, o.pi
    cand = torch.empty(n * pi, dtype=torch.int32, device="cuda")
    score = torch.empty(n * pi, dtype=torch.int64, device="cuda")
    mate = torch.empty(n, dtype=torch.int32, device="cuda")
    st, pairs = hp.hp_debug_coarsen_level(n, g.num_hedges, d["off"].data_ptr(), d["pins"].data_ptr(),
                                          d["src"].data_ptr(), d["w"].data_ptr(), d["size"].data_ptr(), omega, delta,
                                          seed, level, ctypes.byref(o), cand.data_ptr(), score.data_ptr(),
                                          mate.data_ptr())
    assert st == hp.HP_OK, hp.hp_last_error()
    return (cand.cpu().numpy().reshape(n, pi), score.cpu().numpy().view(np.uint64).reshape(n, pi),
            mate.cpu().numpy(), pairs)


def gpu_refine(torch, g, size, rho, nparts, second_half, omega, delta, **opts):
    d = level_arrays(torch, g, size)
    o = hp.options(**opts)
    n = g.num_nodes
    r = dev(torch, np.asarray(rho, np.int32)).clone()
    b = [torch.empty(max(n, 1), dtype=t, device="cuda") for t in (torch.int32, torch.int32, torch.int32,
                                                                    torch.int64, torch.int32, torch.int64)]
    st, m, k, bg = hp.hp_debug_refine_rep(n, g.num_hedges, d["off"].data_ptr(), d["pins"].data_ptr(),
                                          d["src"].data_ptr(), d["w"].data_ptr(), d["size"].data_ptr(), r.data_ptr(),
                                          nparts, int(second_half), omega, delta, ctypes.byref(o),
                                          *[x.data_ptr() for x in b])
    assert st == hp.HP_OK, hp.hp_last_error()
    node, src, dst, gain, seq, gseq = [x.cpu().numpy()[:m] for x in b]
    return dict(node=node, src=src, dst=dst, gain=gain, seq=seq, gseq=gseq, m=m, k=k, best=bg,
                rho=r.cpu().numpy())


GRAPHS = [
    dict(n=40, e=50, max_size=6, seed=1),
    dict(n=200, e=260, max_size=10, seed=2, multi_src=True),
    dict(n=500, e=450, max_size=25, seed=3, weights=True, isolated=20),
    dict(n=1500, e=1400, max_size=60, seed=4, multi_src=True),
]


@pytest.mark.parametrize("spec", GRAPHS)
@pytest.mark.parametrize("pi,permille", [(1, 100), (4, 100), (4, 0), (7, 0), (16, 30)])
def test_coarsen_level_step(torch, spec, pi, permille):
    g = inputs.random_hypergraph(**spec)
    rng = np.random.default_rng(spec["seed"])
    size = rng.integers(1, 4, g.num_nodes).astype(np.int32)
    omega, delta, seed, level = 6, 25, 9, 3
    cand, score, mate, pairs = gpu_coarsen(torch, g, size, omega, delta, seed, level, pi=pi, noise_permille=permille)
    ocand, oscore = oracle.propose(g, size, omega, delta, seed, level, pi, permille)
    assert np.array_equal(cand, ocand)
    assert np.array_equal(score[ocand >= 0], oscore[ocand >= 0])
    p0, m0 = oracle.pair_isolated(g, size, omega, delta, ocand, np.full(g.num_nodes, -1, np.int32))
    p1, m1 = oracle.match_all(ocand, oscore, m0)
    assert pairs == p0 + p1
    assert np.array_equal(mate, m1)


@pytest.mark.parametrize("spec", GRAPHS)
@pytest.mark.parametrize("cap", [64, 128])
def test_coarsen_level_step_overflow(torch, spec, cap):
    g = inputs.random_hypergraph(**spec)
    size = np.ones(g.num_nodes, np.int32)
    cand, score, mate, pairs = gpu_coarsen(torch, g, size, 4, 40, 1, 0, debug_table_cap=cap)
    ocand, oscore = oracle.propose(g, size, 4, 40, 1, 0, 4, 100)
    assert np.array_equal(cand, ocand)


@pytest.mark.parametrize("spec", GRAPHS)
@pytest.mark.parametrize("second_half", [0, 1])
@pytest.mark.parametrize("window,rounds", [(256, 16), (3, 2), (1, 1), (8, 0)])
def test_refine_rep_step(torch, spec, second_half, window, rounds):
    g = inputs.random_hypergraph(**spec)
    n = g.num_nodes
    rng = np.random.default_rng(spec["seed"] + 17)
    nparts = max(2, n // 8)
    rho = rng.integers(0, nparts, n).astype(np.int32)
    size = rng.integers(1, 3, n).astype(np.int32)
    omega = int(np.bincount(rho, weights=size, minlength=nparts).max()) + 2
    ins = [set() for _ in range(n)]
    for e, (s, d) in enumerate(g.edges()):
        for v in d:
            ins[v].add(e)
    delta = max(len(set().union(*[ins[v] for v in range(n) if rho[v] == p])) for p in range(nparts)) + 3
    r = gpu_refine(torch, g, size, rho, nparts, second_half, omega, delta, chain_window=window, chain_rounds=rounds)
    node, src, dst, gain = oracle.propose_moves(g, size, rho, nparts, omega, second_half)
    assert r["m"] == len(node)
    assert np.array_equal(r["node"], node) and np.array_equal(r["src"], src)
    assert np.array_equal(r["dst"], dst) and np.array_equal(r["gain"], gain)
    seq = oracle.sequence(g, size, nparts, node, src, dst, gain, window, rounds)
    assert np.array_equal(r["seq"], seq)
    gseq, k, bg = oracle.inseq_and_prefix(g, size, rho, nparts, node[seq], dst[seq], omega, delta)
    assert np.array_equal(r["gseq"], gseq)
    assert (r["k"], r["best"]) == (k, bg)
    k2, rho2 = oracle.refine_rep(g, size, rho, nparts, second_half, omega, delta, window, rounds)
    assert r["k"] == k2 and np.array_equal(r["rho"], rho2)
