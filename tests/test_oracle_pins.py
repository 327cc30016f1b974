"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one step of the oracle against something other than the
oracle itself: hand-derived values (tests/golden/*.json), brute force on tiny
inputs computed by a different route (set algebra, exhaustive enumeration),
a textbook routine (networkx maximum-weight matching), closed forms and the
invariants the paper states (two-cycle pseudo-forest of Sec. V-A, telescoping
of in-sequence gains of Sec. VI-C, Score/Conn duality of Sec. III).
"""
import itertools
import json
import os

import networkx as nx
import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def hg_from(d):
    return inputs.Hypergraph(d["num_nodes"], np.array(d["offsets"], np.int32), np.array(d["pins"], np.int32),
                             np.array(d["src_counts"], np.int32) if "src_counts" in d else None)


def edge_list(g):
    """[(src set, dst set, w)] straight from the CSR definition (Sec. II-A)."""
    out = []
    for e, (s, d) in enumerate(g.edges()):
        w = 1 if g.weights is None else int(g.weights[e])
        out.append((set(s), set(d), w))
    return out


def conn_bf(g, rho):
    """Eq. 1 by set comprehension."""
    return sum(w * (len({int(rho[v]) for v in s | d}) - 1) for s, d, w in edge_list(g))


def inbound_sets(g):
    ins = [set() for _ in range(g.num_nodes)]
    for e, (s, d, w) in enumerate(edge_list(g)):
        for v in d:
            ins[v].add(e)
    return ins


def q_of(size, w=1):
    return (w << 24) // size


SMALL_GRAPHS = [
    dict(n=12, e=10, max_size=5, seed=1),
    dict(n=20, e=30, max_size=6, seed=2, multi_src=True),
    dict(n=16, e=25, max_size=4, seed=3, weights=True),
    dict(n=25, e=20, max_size=8, seed=4, multi_src=True, weights=True, isolated=3),
]


# ---------------------------------------------------------------- Eq. 5 / inter
def test_golden_eta_inter():
    d = load("eta_small.json")
    g = hg_from(d)
    k, eta0, inter, cap = oracle.node_histogram(g, d["node"])
    assert k == d["num_neighbours"]
    assert eta0.tolist() == d["eta0"]
    assert inter.tolist() == d["inter"]
    assert cap == d["noise_cap"]


@pytest.mark.parametrize("spec", SMALL_GRAPHS)
def test_eta_inter_brute_force(spec):
    g = inputs.random_hypergraph(**spec)
    E = edge_list(g)
    ins = inbound_sets(g)
    for v in range(g.num_nodes):
        k, eta0, inter, _ = oracle.node_histogram(g, v)
        nbrs = set()
        exp = np.zeros(g.num_nodes, dtype=np.uint64)
        for s, dd, w in E:
            e_all = s | dd
            if v in e_all:
                for m in e_all - {v}:
                    exp[m] += q_of(len(e_all), w)
                nbrs |= e_all - {v}
        assert k == len(nbrs)
        assert np.array_equal(eta0, exp)
        for m in range(g.num_nodes):
            assert inter[m] == (len(ins[v] & ins[m]) if m in nbrs else 0)


def test_eta_symmetric_and_closed_form():
    # one hyperedge holding every node: eta(n, m) = q(e) for all pairs
    n = 9
    g = inputs.Hypergraph(n, np.array([0, n], np.int32), np.arange(n, dtype=np.int32))
    for v in range(n):
        k, eta0, inter, _ = oracle.node_histogram(g, v)
        assert k == n - 1
        assert all(int(eta0[m]) == q_of(n) for m in range(n) if m != v)
        # node 0 is the source, every other node a destination
        assert all(int(inter[m]) == (1 if v > 0 and m > 0 else 0) for m in range(n) if m != v)
    # symmetry on irregular graphs with weights and multi-source hyperedges
    g = inputs.random_hypergraph(30, 40, 7, seed=9, multi_src=True, weights=True)
    H = np.stack([oracle.node_histogram(g, v)[1] for v in range(30)])
    I = np.stack([oracle.node_histogram(g, v)[2] for v in range(30)])
    assert np.array_equal(H, H.T) and np.array_equal(I, I.T)


def test_noise_symmetric_capped_uniform():
    cap = 1000
    vals = []
    for a in range(40):
        for b in range(40):
            x = oracle.pair_noise(7, 3, a, b, cap)
            assert x == oracle.pair_noise(7, 3, b, a, cap)
            assert 0 <= x <= cap
            vals.append(x)
    vals = np.array(vals)
    assert abs(vals.mean() - cap / 2) < 40          # roughly uniform on [0, cap]
    assert oracle.pair_noise(7, 3, 1, 2, 0) == 0
    assert oracle.pair_noise(7, 3, 1, 2, cap) != oracle.pair_noise(8, 3, 1, 2, cap) or \
        oracle.pair_noise(7, 4, 1, 2, cap) != oracle.pair_noise(7, 3, 1, 2, cap)


# ------------------------------------------------------------ Eq. 6, top-Pi
@pytest.mark.parametrize("spec", SMALL_GRAPHS)
@pytest.mark.parametrize("omega,delta", [(3, 100), (100, 4), (2, 2)])
@pytest.mark.parametrize("permille", [100, 0])
def test_proposal_matches_definition(spec, omega, delta, permille):
    """Eq. 6; without noise (permille 0) equal eta values are frequent, so the
    max-id tie rule is exercised."""
    g = inputs.random_hypergraph(**spec)
    rng = np.random.default_rng(5)
    size = rng.integers(1, 3, g.num_nodes).astype(np.int32)
    pi, seed, level = 3, 11, 2
    cand, score = oracle.propose(g, size, omega, delta, seed, level, pi, permille)
    E = edge_list(g)
    ins = inbound_sets(g)
    qs = [q_of(len(s | d), w) for s, d, w in E]
    cap = (sum(qs) // len(qs)) * permille // 1000
    for v in range(g.num_nodes):
        eta = {}
        for (s, d, w), q in zip(E, qs):
            if v in s | d:
                for m in (s | d) - {v}:
                    eta[m] = eta.get(m, 0) + q
        valid = [m for m in eta if size[v] + size[m] <= omega and len(ins[v] | ins[m]) <= delta]
        keyed = sorted(((eta[m] + oracle.pair_noise(seed, level, v, m, cap), m) for m in valid), reverse=True)
        exp = keyed[:pi]
        got = [(int(score[v, i]), int(cand[v, i])) for i in range(pi) if cand[v, i] >= 0]
        assert got == exp


def _round_targets(cand, score, mate):
    n, pi = cand.shape
    t = np.full(n, -1, np.int32)
    s = np.zeros(n, np.uint64)
    for v in range(n):
        if mate[v] >= 0:
            continue
        for i in range(pi):
            c = cand[v, i]
            if c < 0:
                break
            if mate[c] < 0:
                t[v], s[v] = c, score[v, i]
                break
    return t, s


def _cycles(target):
    """lengths of the cycles of the functional graph v -> target[v]."""
    n = len(target)
    state = np.zeros(n, np.int8)
    out = []
    for v in range(n):
        path, u = [], v
        while u >= 0 and state[u] == 0:
            state[u] = 1
            path.append(u)
            u = target[u]
        if u >= 0 and state[u] == 1:
            out.append(len(path) - path.index(u))
        for x in path:
            state[x] = 2
    return out


@pytest.mark.parametrize("seed", range(6))
def test_proposal_graph_only_two_cycles(seed):
    """Sec. V-A: with symmetric eta and max-id ties every cycle has length 2,
    in every one of the Pi rounds."""
    g = inputs.random_hypergraph(60, 80, 6, seed=seed, multi_src=seed % 2 == 1)
    size = np.ones(60, np.int32)
    cand, score = oracle.propose(g, size, 4, 50, seed, 0, 4, permille=0 if seed < 3 else 100)
    mate = np.full(60, -1, np.int32)
    for r in range(4):
        t, s = _round_targets(cand, score, mate)
        assert all(c == 2 for c in _cycles(t))
        _, rm = oracle.match_round(t, s)
        mate = np.where(rm >= 0, rm, mate).astype(np.int32)


# ------------------------------------------------------- Eq. 7-12 matching
def test_golden_matching():
    for case in load("matching_dp.json")["cases"]:
        pairs, mate = oracle.match_round(np.array(case["target"], np.int32), np.array(case["score"], np.uint64))
        assert mate.tolist() == case["mate"], case["name"]
        w = sum(case["score"][v] for v in range(len(mate)) if mate[v] == case["target"][v] and mate[v] >= 0
                and (case["target"][mate[v]] != v or v < mate[v]))
        assert w == case["weight"]


def _random_pseudoforest(n, rng, ties=False):
    """Each node targets its best neighbour by (w, id) in a random symmetric
    weighted graph: the proposal-graph structure of Eq. 6."""
    W = np.zeros((n, n), np.int64)
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < 0.3:
                W[a, b] = W[b, a] = int(rng.integers(1, 4 if ties else 1000))
    target = np.full(n, -1, np.int32)
    score = np.zeros(n, np.uint64)
    for v in range(n):
        best = None
        for m in range(n):
            if W[v, m] > 0 and (best is None or (W[v, m], m) > (W[v, best], best)):
                best = m
        if best is not None:
            target[v], score[v] = best, W[v, best]
    return target, score


def _matching_weight(target, score, mate):
    w = 0
    for v in range(len(mate)):
        m = mate[v]
        if m < 0 or v > m:
            continue
        assert mate[m] == v
        # the pair must be a proposal edge
        if target[v] == m:
            w += int(score[v])
        else:
            assert target[m] == v
            w += int(score[m])
    return w


@pytest.mark.parametrize("seed", range(12))
def test_matching_is_maximum_weight(seed):
    rng = np.random.default_rng(seed)
    n = 80 if seed % 2 else 12
    target, score = _random_pseudoforest(n, rng, ties=seed % 3 == 0)
    pairs, mate = oracle.match_round(target, score)
    got = _matching_weight(target, score, mate)
    G = nx.Graph()
    for v in range(n):
        if target[v] >= 0:
            a, b = sorted((v, int(target[v])))
            G.add_edge(a, b, weight=int(score[v]))
    best = nx.max_weight_matching(G)
    exp = sum(G[a][b]["weight"] for a, b in best)
    assert got == exp
    assert pairs == sum(1 for v in range(n) if mate[v] > v)


# ------------------------------------------------- isolated-node pairing
def test_isolated_pairing():
    # 6 nodes without hyperedges (sizes 1..3), plus one connected pair
    g = inputs.Hypergraph(8, np.array([0, 2], np.int32), np.array([6, 7], np.int32))
    size = np.array([3, 1, 2, 1, 2, 3, 1, 1], np.int32)
    cand, score = oracle.propose(g, size, 4, 10, 0, 0, 4)
    assert (cand[:6, 0] == -1).all() and cand[6, 0] == 7
    pairs, mate = oracle.pair_isolated(g, size, 4, 10, cand, np.full(8, -1, np.int32))
    # every pair fits, nodes with a valid neighbour are left to the matching,
    # and at most one fitting isolated node stays single
    for v in range(6):
        if mate[v] >= 0:
            assert size[v] + size[mate[v]] <= 4 and mate[mate[v]] == v
    assert mate[6] == -1 and mate[7] == -1
    assert pairs == 3
    # closed form: k unit-size isolated nodes with no inbound edges -> k//2 pairs
    for k in (1, 2, 7, 10):
        g = inputs.Hypergraph(k, np.array([0], np.int32), np.zeros(0, np.int32))
        cand, _ = oracle.propose(g, np.ones(k, np.int32), 2, 0, 0, 0, 4)
        p, _ = oracle.pair_isolated(g, np.ones(k, np.int32), 2, 0, cand, np.full(k, -1, np.int32))
        assert p == k // 2


# -------------------------------------------------------- Sec. V-E contraction
@pytest.mark.parametrize("spec", SMALL_GRAPHS)
def test_contraction_matches_set_definition(spec):
    g = inputs.random_hypergraph(**spec)
    n = g.num_nodes
    rng = np.random.default_rng(3)
    perm = rng.permutation(n)
    mate = np.full(n, -1, np.int32)
    for i in range(0, n - 1, 3):                  # pair 2 of every 3 nodes
        a, b = perm[i], perm[i + 1]
        mate[a], mate[b] = b, a
    size = rng.integers(1, 4, n).astype(np.int32)
    gamma, csize, coff, cpins, cnsrc = oracle.contract(g, size, mate)
    # gamma: rank of the cluster's smallest member
    reps = sorted(v for v in range(n) if mate[v] < 0 or v < mate[v])
    for v in range(n):
        assert gamma[v] == reps.index(min(v, mate[v]) if mate[v] >= 0 else v)
    assert csize.sum() == size.sum()
    for v in range(n):
        assert csize[gamma[v]] == size[v] + (size[mate[v]] if mate[v] >= 0 else 0)
    cg = inputs.Hypergraph(len(csize), coff, cpins, cnsrc)
    for (s, d, w), (cs, cd) in zip(edge_list(g), cg.edges()):
        dd = {int(gamma[v]) for v in d}
        ss = {int(gamma[v]) for v in s} - dd
        assert set(cd) == dd and len(cd) == len(dd)
        assert set(cs) == ss and len(cs) == len(ss)
    # Score/Conn duality (Sec. III): Score(gamma) + Conn(gamma) = sum w(|e| - 1)
    score = sum(w * (len(s | d) - len({int(gamma[v]) for v in s | d})) for s, d, w in edge_list(g))
    conn, _ = oracle.objective(g, gamma, len(csize))
    assert score + conn == sum(w * (len(s | d) - 1) for s, d, w in edge_list(g))


def test_objective_closed_forms():
    g = inputs.random_hypergraph(30, 40, 6, seed=4, weights=True)
    E = edge_list(g)
    total = sum(w * (len(s | d) - 1) for s, d, w in E)
    assert oracle.objective(g, np.zeros(30, np.int32), 1) == (0, 0)
    c, cn = oracle.objective(g, np.arange(30, dtype=np.int32), 30)
    assert c == total and cn == sum(w for s, d, w in E if len(s | d) > 1)
    rho = np.random.default_rng(1).integers(0, 4, 30).astype(np.int32)
    assert oracle.objective(g, rho, 4)[0] == conn_bf(g, rho)


# ------------------------------------------------------ Eq. 13 move gains
@pytest.mark.parametrize("spec", SMALL_GRAPHS)
@pytest.mark.parametrize("second_half", [0, 1])
def test_move_gain_is_connectivity_change(spec, second_half):
    g = inputs.random_hypergraph(**spec)
    n = g.num_nodes
    rng = np.random.default_rng(7)
    nparts = 5
    rho = rng.integers(0, nparts, n).astype(np.int32)
    size = rng.integers(1, 3, n).astype(np.int32)
    omega = int(size.sum() // 3)
    node, src, dst, gain = oracle.propose_moves(g, size, rho, nparts, omega, second_half)
    base = conn_bf(g, rho)
    psize = np.bincount(rho, weights=size, minlength=nparts)
    E = edge_list(g)
    proposed = {int(v): (int(d), int(x)) for v, d, x in zip(node, dst, gain)}
    for v in range(n):
        adj = {int(rho[m]) for s, d, w in E if v in s | d for m in s | d} - {int(rho[v])}
        best = None
        for p in adj:
            if second_half and size[v] + psize[p] > omega:
                continue
            r2 = rho.copy()
            r2[v] = p
            gp = base - conn_bf(g, r2)
            if best is None or (gp, p) > best:
                best = (gp, p)
        if best is not None and best[0] > 0:
            assert proposed.get(v) == (best[1], best[0])
        else:
            assert v not in proposed
    # sorted by (p_s asc, gain desc, node asc)
    keys = [(int(s), -int(x), int(v)) for v, s, x in zip(node, src, gain)]
    assert keys == sorted(keys)


# -------------------------------------- Eq. 14-15 in-sequence gains + prefix
def test_golden_inseq():
    d = load("inseq_small.json")
    g = hg_from(d)
    rho = np.array(d["rho"], np.int32)
    gseq, k, bg = oracle.inseq_and_prefix(g, np.ones(4, np.int32), rho, d["nparts"],
                                          np.array(d["sequence_nodes"], np.int32),
                                          np.array(d["sequence_dst"], np.int32), 100, 100)
    assert gseq.tolist() == d["gseq"]
    assert conn_bf(g, rho) == d["conn_before"]
    node, src, dst, gain = oracle.propose_moves(g, np.ones(4, np.int32), rho, 2, 100, 0)
    assert dict(zip(node.tolist(), gain.tolist()))[1] == d["isolation_gain_of_node1"]


@pytest.mark.parametrize("seed", range(8))
def test_inseq_gains_telescope_and_best_prefix(seed):
    g = inputs.random_hypergraph(30, 45, 6, seed=seed, multi_src=seed % 2 == 0, weights=seed % 3 == 0)
    n = g.num_nodes
    rng = np.random.default_rng(seed)
    nparts = 4
    rho = rng.integers(0, nparts, n).astype(np.int32)
    size = rng.integers(1, 3, n).astype(np.int32)
    nodes = rng.permutation(n)[:15].astype(np.int32)
    dst = np.array([(rho[v] + rng.integers(1, nparts)) % nparts for v in nodes], np.int32)
    ins = inbound_sets(g)
    psize0 = np.bincount(rho, weights=size, minlength=nparts)
    omega = int(psize0.max())
    D0 = [len(set().union(*[ins[v] for v in range(n) if rho[v] == p])) for p in range(nparts)]
    delta = int(max(D0))
    gseq, k, bg = oracle.inseq_and_prefix(g, size, rho, nparts, nodes, dst, omega, delta)
    r = rho.copy()
    c0 = conn_bf(g, rho)
    cum, best, bestk = 0, 0, 0
    for i, (v, d) in enumerate(zip(nodes, dst)):
        r[v] = d
        cum += int(gseq[i])
        assert cum == c0 - conn_bf(g, r)            # exact telescoping
        # validity recomputed from scratch
        ok = all(sum(size[u] for u in range(n) if r[u] == p) <= omega and
                 len(set().union(*[ins[u] for u in range(n) if r[u] == p])) <= delta for p in range(nparts))
        if ok and cum >= best:
            best, bestk = cum, i + 1
    assert (k, bg) == ((bestk, best) if best > 0 else (0, best))


# ---------------------------------------------------------- Sec. VI-C chains
@pytest.mark.parametrize("seed", range(6))
def test_sequence_structure(seed):
    g = inputs.random_hypergraph(60, 90, 5, seed=seed)
    n = g.num_nodes
    rng = np.random.default_rng(seed)
    nparts = 6
    rho = rng.integers(0, nparts, n).astype(np.int32)
    size = np.ones(n, np.int32)
    node, src, dst, gain = oracle.propose_moves(g, size, rho, nparts, n, 0)
    M = len(node)
    seq = oracle.sequence(g, size, nparts, node, src, dst, gain)
    assert sorted(seq.tolist()) == list(range(M))
    # the sequence splits into chains whose links join p_d of a move to p_s of
    # the next; chains come in non-increasing order of their total gain
    chains, cur = [], [seq[0]] if M else []
    for a, b in zip(seq[:-1], seq[1:]):
        if dst[a] == src[b]:
            cur.append(b)
        else:
            chains.append(cur)
            cur = [b]
    if cur:
        chains.append(cur)
    # the greedy link split can only merge true chains, so totals of maximal
    # runs need not be sorted; the first move of the sequence heads the
    # highest-gain chain, which is at least the best single move
    if M:
        assert sum(gain[i] for i in chains[0]) >= gain.max()
    # with a window of 1 and one round, each chain has at most 2 moves
    seq1 = oracle.sequence(g, size, nparts, node, src, dst, gain, window=1, rounds=1)
    assert sorted(seq1.tolist()) == list(range(M))
    # no rounds: chains are single moves ordered by (gain desc, node asc)
    seq0 = oracle.sequence(g, size, nparts, node, src, dst, gain, rounds=0)
    assert [(-int(gain[i]), int(node[i])) for i in seq0] == sorted((-int(x), int(v)) for v, x in zip(node, gain))


# --------------------------------------------------------------- end to end
def partitions_of(n):
    """all set partitions of range(n) as label arrays (restricted growth)."""
    def rec(i, labels, k):
        if i == n:
            yield list(labels)
            return
        for c in range(k + 1):
            labels.append(c)
            yield from rec(i + 1, labels, max(k, c + 1))
            labels.pop()
    yield from rec(0, [], 0)


def feasible(g, rho, omega, delta):
    ins = inbound_sets(g)
    for p in set(rho.tolist()):
        members = [v for v in range(g.num_nodes) if rho[v] == p]
        if len(members) > omega or len(set().union(*[ins[v] for v in members])) > delta:
            return False
    return True


@pytest.mark.parametrize("seed", range(10))
def test_end_to_end_vs_brute_force_optimum(seed):
    n = 8
    g = inputs.random_hypergraph(n, 7, 4, seed=100 + seed, multi_src=seed % 2 == 0)
    omega, delta = 3, 4
    r = oracle.partition(g, omega, delta, seed)
    assert r.status == oracle.OK
    assert feasible(g, r.part, omega, delta)
    assert r.stats["connectivity"] == conn_bf(g, r.part)
    opt = min(conn_bf(g, np.array(lab)) for lab in partitions_of(n)
              if feasible(g, np.array(lab), omega, delta))
    assert r.stats["connectivity"] >= opt
    # never worse than leaving every node alone
    assert r.stats["connectivity"] <= conn_bf(g, np.arange(n))


@pytest.mark.parametrize("seed", range(4))
def test_planted_components_reach_zero_connectivity(seed):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(2, 9, 12).tolist()
    g = inputs.planted_components(sizes, edges_per_comp=6, edge_size=3, seed=seed)
    r = oracle.partition(g, 8, 1000, seed)
    assert r.status == oracle.OK
    assert r.stats["connectivity"] == 0
    assert r.stats["violations"] == 0


def test_independent_checker_on_random_snn():
    g = inputs.random_snn(512, 15, seed=3)
    omega, delta = 32, 160
    r = oracle.partition(g, omega, delta, 0)
    assert r.status == oracle.OK
    assert r.stats["connectivity"] == conn_bf(g, r.part)
    assert feasible(g, r.part, omega, delta)
    assert r.stats["violations"] == 0
    # part ids are compact
    assert sorted(set(r.part.tolist())) == list(range(r.stats["num_parts"]))
    # well below the one-pass fill heuristic (fill partitions in id order)
    ins = inbound_sets(g)
    one, p, cur, cur_in = np.zeros(512, np.int32), 0, 0, set()
    for v in range(512):
        if cur + 1 > omega or len(cur_in | ins[v]) > delta:
            p, cur, cur_in = p + 1, 0, set()
        one[v], cur, cur_in = p, cur + 1, cur_in | ins[v]
    assert r.stats["connectivity"] < conn_bf(g, one)


def test_determinism_and_incident_mode():
    g = inputs.random_hypergraph(200, 260, 8, seed=5, multi_src=True)
    a = oracle.partition(g, 16, 60, 1)
    b = oracle.partition(g, 16, 60, 1)
    assert np.array_equal(a.part, b.part) and a.stats == b.stats
    # incident counting == inbound counting with every pin a destination
    c = oracle.partition(g, 16, 60, 1, count_kind=oracle.COUNT_INCIDENT)
    g0 = inputs.Hypergraph(g.num_nodes, g.offsets, g.pins, np.zeros(g.num_hedges, np.int32))
    d = oracle.partition(g0, 16, 60, 1)
    assert np.array_equal(c.part, d.part)
    assert feasible(g0, c.part, 16, 60)


def test_error_statuses():
    g = inputs.random_hypergraph(10, 5, 3, seed=1)
    assert oracle.partition(g, 0, 5).status == oracle.ERR_INVALID_ARG
    bad = inputs.Hypergraph(10, g.offsets, g.pins.copy())
    bad.pins[0] = 10
    assert oracle.partition(bad, 4, 5).status == oracle.ERR_BAD_CSR
    dup = inputs.Hypergraph(3, np.array([0, 2], np.int32), np.array([1, 1], np.int32))
    assert oracle.partition(dup, 4, 5).status == oracle.ERR_BAD_CSR
    empty_edge = inputs.Hypergraph(3, np.array([0, 0], np.int32), np.zeros(0, np.int32))
    assert oracle.partition(empty_edge, 4, 5).status == oracle.ERR_BAD_CSR
    srcbad = inputs.Hypergraph(3, np.array([0, 2], np.int32), np.array([0, 1], np.int32),
                               np.array([3], np.int32))
    assert oracle.partition(srcbad, 4, 5).status == oracle.ERR_BAD_CSR
    star = inputs.Hypergraph(4, np.array([0, 2, 4, 6], np.int32), np.array([0, 3, 1, 3, 2, 3], np.int32))
    assert oracle.partition(star, 4, 2).status == oracle.ERR_INFEASIBLE
    assert oracle.partition(star, 4, 3).status == oracle.OK
    w = inputs.Hypergraph(4, star.offsets, star.pins, None, np.array([1, 0, 1], np.int32))
    assert oracle.partition(w, 4, 3).status == oracle.ERR_INVALID_ARG
    empty = inputs.Hypergraph(0, np.array([0], np.int32), np.zeros(0, np.int32))
    r = oracle.partition(empty, 4, 3)
    assert r.status == oracle.OK and r.stats["num_parts"] == 0


def all_set_partitions(n):
    """Every set partition of range(n) as a label array (restricted growth
    strings: label i is at most 1 + the largest label before it), built
    column by column: Bell(n) rows."""
    rows = np.zeros((1, 1), dtype=np.int8)
    for _ in range(1, n):
        mx = rows.max(axis=1).astype(np.int64)
        cnt = mx + 2
        rep = np.repeat(rows, cnt, axis=0)
        nxt = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        rows = np.concatenate([rep, nxt[:, None].astype(np.int8)], axis=1)
    return rows


def brute_force_optimum(g, omega, delta):
    """Minimum connectivity (Eq. 1) over every feasible set partition, by
    exhaustive enumeration (vectorised over the partitions)."""
    n = g.num_nodes
    lab = all_set_partitions(n).astype(np.int64)
    w = np.ones(g.num_hedges, dtype=np.int64) if g.weights is None else g.weights.astype(np.int64)
    conn = np.zeros(lab.shape[0], dtype=np.int64)
    inmask = np.zeros(n, dtype=np.int64)
    for e, (src, dst) in enumerate(g.edges()):
        pins = list(src) + list(dst)
        s = np.sort(lab[:, pins], axis=1)
        lam = 1 + (np.diff(s, axis=1) != 0).sum(axis=1)
        conn += w[e] * (lam - 1)
        for v in dst:
            inmask[v] |= np.int64(1) << e
    ok = np.ones(lab.shape[0], dtype=bool)
    for p in range(n):
        members = lab == p
        ok &= members.sum(axis=1) <= omega
        m = np.bitwise_or.reduce(np.where(members, inmask[None, :], 0), axis=1)
        bits = np.zeros_like(m)
        for b in range(g.num_hedges):
            bits += (m >> b) & 1
        ok &= bits <= delta
    return int(conn[ok].min()), int(ok.sum())


def test_set_partition_enumeration_counts():
    # Bell numbers B(1..8) and B(12)
    assert [all_set_partitions(n).shape[0] for n in range(1, 9)] == [1, 2, 5, 15, 52, 203, 877, 4140]
    assert all_set_partitions(12).shape[0] == 4213597


@pytest.mark.parametrize("seed", range(3))
def test_end_to_end_vs_brute_force_optimum_12_nodes(seed):
    """12 nodes: the oracle's result is feasible, its connectivity is the
    one recomputed by set comprehension, and no feasible partition of the
    4,213,597 is better than the exhaustive optimum it is compared to."""
    n = 12
    g = inputs.random_hypergraph(n, 9, 5, seed=300 + seed, multi_src=seed == 1, weights=seed == 2)
    omega, delta = 4, 5
    r = oracle.partition(g, omega, delta, seed)
    assert r.status == oracle.OK
    assert feasible(g, r.part, omega, delta)
    assert r.stats["connectivity"] == conn_bf(g, r.part)
    opt, nfeas = brute_force_optimum(g, omega, delta)
    assert nfeas > 0
    assert opt <= r.stats["connectivity"] <= conn_bf(g, np.arange(n))
