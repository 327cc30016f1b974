"""Pins of the oracle's learned merge priority (a growth of Sec. V-C that the
paper does not have: the top-K candidate lists by (eta, id), pairs kept only
when mutual, C(n) = top Pi of those by (s, eta, id), s an integer MLP of
sixteen symmetric pair features; the matching weight stays eta).

What fixes it from outside the oracle:
* the MLP on hand-built models whose score has a closed form (one path
  through the network, the clamp at 255, the floor shift, ReLU at 0);
* the log code at values worked out by hand;
* the features against a brute-force recount from the hyperedge lists;
* symmetry of the features and of the score;
* with a constant model and K at least every node's number of valid
  neighbours, the learned priority is the plain one: same C(n), same
  partition;
* the proposal graph of every round has no cycle longer than two;
* C(n) against a brute-force selection from the pinned scores.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import inputs


def zero_model():
    return inputs.constant_merge_model(0)


# ---------------------------------------------------------------- MLP closed forms
def test_mlp_single_path():
    # s = b3 + w3[7] * a2[7], a2[7] = w2[7][5] * a1[5], a1[5] = f[3]
    m = zero_model()
    m.w1[5, 3] = 1
    m.w2[7, 5] = 1
    m.w3[7] = 2
    m.b3 = -11
    f = np.zeros((4, 16), np.uint8)
    f[:, 3] = [0, 1, 200, 255]
    f[:, 4] = 99   # not on the path
    assert list(oracle.mlp_scores(f, m)) == [-11, -9, 389, 499]


def test_mlp_clamp_shift_relu():
    m = zero_model()
    m.w1[0, 0] = 127
    m.w1[1, 0] = -127
    m.b1[2] = 1000   # a1[2] = min(255, 1000 >> s1)
    m.w2[0, 0] = 1   # a2[0] = a1[0]
    m.w2[1, 1] = 1   # a2[1] = a1[1] = 0 (ReLU)
    m.w2[2, 2] = 1   # a2[2] = a1[2]
    m.w3[0], m.w3[1], m.w3[2] = 1, 50, 100
    for s1, f0, want in [(0, 255, 255 + 100 * 255),   # 127*255 and 1000 clamp at 255
                         (8, 255, 126 + 100 * 3),     # 32385 >> 8, 1000 >> 8
                         (8, 3, 1 + 100 * 3),         # 381 >> 8
                         (30, 255, 0)]:
        m.shift1 = s1
        f = np.zeros((1, 16), np.uint8)
        f[0, 0] = f0
        assert oracle.mlp_scores(f, m)[0] == want, (s1, f0)


def test_mlp_second_shift_and_bias():
    m = zero_model()
    m.b1[:] = 40              # a1 = 40 everywhere
    m.w2[3, :] = 1            # h2[3] = 64 * 40 + b2[3]
    m.b2[3] = -60
    m.shift2 = 4              # a2[3] = (2560 - 60) >> 4 = 156
    m.w3[3] = -3
    m.b3 = 5
    assert oracle.mlp_scores(np.zeros((1, 16), np.uint8), m)[0] == 5 - 3 * 156


def test_mlp_monotone_for_nonnegative_weights():
    m = inputs.random_merge_model(3)
    for a in (m.w1, m.w2, m.w3):
        np.abs(a, out=a)
    rng = np.random.default_rng(1)
    f = rng.integers(0, 200, size=(200, 16)).astype(np.uint8)
    g = f.copy()
    g[:, rng.integers(0, 16)] += 50
    assert np.all(oracle.mlp_scores(g, m) >= oracle.mlp_scores(f, m))


def test_invalid_models_rejected():
    for mut in (lambda m: m.w1.__setitem__((0, 0), -128), lambda m: setattr(m, "shift1", 31),
                lambda m: setattr(m, "b3", 2**30 + 1), lambda m: m.b2.__setitem__(1, -(2**30) - 1)):
        m = inputs.random_merge_model(0)
        mut(m)
        with pytest.raises(ValueError):
            oracle.mlp_scores(np.zeros((1, 16), np.uint8), m)


# ---------------------------------------------------------------- log code
def test_log_code_values():
    # 0 -> 0; else 1 + 4 floor(log2 x) + the two bits after the leading one
    want = {0: 0, 1: 1, 2: 5, 3: 7, 4: 9, 5: 10, 6: 11, 7: 12, 8: 13, 12: 15, 1 << 20: 81,
            (1 << 20) + (1 << 19): 83, 1 << 62: 249, 1 << 63: 253, 2**64 - 1: 255}
    for x, c in want.items():
        assert oracle.log_code(x) == c, x
    xs = sorted(set(np.random.default_rng(0).integers(0, 2**62, size=500).tolist()) | set(range(300)))
    codes = [oracle.log_code(x) for x in xs]
    assert codes == sorted(codes)


# ---------------------------------------------------------------- features
def _level(g, omega, delta, K, seed=0, level=0, size=None):
    size = np.ones(g.num_nodes, np.int32) if size is None else size
    candK, csK = oracle.propose(g, size, omega, delta, seed=seed, level=level, pi=K)
    return size, candK, csK


def _sets(g):
    n = g.num_nodes
    nsrc = g.src_counts if g.src_counts is not None else np.ones(g.num_hedges, np.int32)
    I = [set() for _ in range(n)]
    In = [set() for _ in range(n)]
    for e in range(g.num_hedges):
        row = g.pins[g.offsets[e]:g.offsets[e + 1]]
        for j, v in enumerate(row):
            I[v].add(e)
            if j >= nsrc[e]:
                In[v].add(e)
    return I, In


def _lc(x):
    x = int(x)
    if x == 0:
        return 0
    b = x.bit_length() - 1
    top3 = x >> (b - 2) if b >= 2 else x << (2 - b)
    return min(255, 1 + 4 * b + (top3 & 3))


@pytest.mark.parametrize("seed,incident", [(0, False), (1, False), (2, False), (3, True)])
def test_features_brute_force(seed, incident):
    g = inputs.random_hypergraph(60, 90, 7, seed=seed, multi_src=True)
    if incident:   # every pin a destination: in(v) = I(v)
        g = inputs.Hypergraph(num_nodes=g.num_nodes, offsets=g.offsets, pins=g.pins,
                              src_counts=np.zeros(g.num_hedges, np.int32))
    rng = np.random.default_rng(seed)
    size = rng.integers(1, 4, size=g.num_nodes).astype(np.int32)
    omega, delta, K, level = 9, 14, 8, 3
    size, candK, csK = _level(g, omega, delta, K, seed=seed, level=level, size=size)
    feat, rank, cand, cs = oracle.learned_level(g, size, omega, delta, level, candK.ravel(), csK.ravel(), 4,
                                                inputs.random_merge_model(seed))
    I, In = _sets(g)
    n = g.num_nodes
    mutual = 0
    for v in range(n):
        for j in range(K):
            m = candK[v, j]
            p = v * K + j
            rm = [i for i in range(K) if candK[m, i] == v] if m >= 0 else []
            assert rank[p] == (rm[0] if rm else -1)
            if not rm:
                assert not feat[p].any()
                continue
            mutual += 1
            sh, it = len(I[v] & I[m]), len(In[v] & In[m])
            uni = len(In[v]) + len(In[m]) - it
            sv, sm = int(size[v]), int(size[m])
            dv, dm = len(I[v]), len(I[m])
            iv, im = len(In[v]), len(In[m])
            want = [_lc(csK[v, j]), _lc(sh), _lc(it), _lc(min(sv, sm)), _lc(max(sv, sm)), _lc(min(iv, im)),
                    _lc(max(iv, im)), _lc(min(dv, dm)), _lc(max(dv, dm)), 255 * (sv + sm) // omega,
                    255 * uni // delta, level, 255 * it // uni if uni else 0, min(j, rm[0]), max(j, rm[0]),
                    _lc(iv + im)]
            assert list(feat[p]) == want, (v, m)
    assert mutual > 50


def test_features_and_scores_symmetric():
    g = inputs.random_snn(300, 11, seed=4)
    omega, delta, K = 16, 64, 16
    size, candK, csK = _level(g, omega, delta, K)
    model = inputs.random_merge_model(9)
    feat, rank, _, _ = oracle.learned_level(g, size, omega, delta, 0, candK.ravel(), csK.ravel(), 4, model)
    s = oracle.mlp_scores(feat, model)
    checked = 0
    for p in np.nonzero(rank >= 0)[0]:
        v, j = divmod(int(p), K)
        m = candK[v, j]
        q = m * K + rank[p]
        assert candK[m, rank[p]] == v and rank[q] == j
        assert np.array_equal(feat[p], feat[q]) and s[p] == s[q]
        checked += 1
    assert checked > 500


# ---------------------------------------------------------------- selection
def test_selection_brute_force():
    g = inputs.random_snn(200, 9, seed=7)
    omega, delta, K, pi = 12, 48, 12, 4
    size, candK, csK = _level(g, omega, delta, K, seed=3)
    model = inputs.random_merge_model(5)
    feat, rank, cand, cs = oracle.learned_level(g, size, omega, delta, 0, candK.ravel(), csK.ravel(), pi, model)
    s = oracle.mlp_scores(feat, model)
    cand, cs = cand.reshape(-1, pi), cs.reshape(-1, pi)
    for v in range(g.num_nodes):
        keys = [(int(s[v * K + j]), int(csK[v, j]), int(candK[v, j])) for j in range(K) if rank[v * K + j] >= 0]
        keys.sort(reverse=True)
        want = [k[2] for k in keys[:pi]] + [-1] * (pi - min(pi, len(keys)))
        assert list(cand[v]) == want
        assert list(cs[v][: len(keys[:pi])]) == [k[1] for k in keys[:pi]]


@pytest.mark.parametrize("seed", range(6))
def test_proposal_graph_has_only_two_cycles(seed):
    g = inputs.random_snn(400, 13, seed=seed)
    omega, delta, K, pi = 8, 40, 16, 4
    size, candK, csK = _level(g, omega, delta, K, seed=seed)
    model = inputs.random_merge_model(100 + seed)
    _, _, cand, _ = oracle.learned_level(g, size, omega, delta, 0, candK.ravel(), csK.ravel(), pi, model)
    cand = cand.reshape(-1, pi)
    n = g.num_nodes
    mate = np.full(n, -1)
    rng = np.random.default_rng(seed)
    for r in range(pi):
        # any set of matched nodes: the targets of the rest must still close only 2-cycles
        tgt = np.full(n, -1)
        for v in range(n):
            if mate[v] < 0:
                for c in cand[v]:
                    if c >= 0 and mate[c] < 0:
                        tgt[v] = c
                        break
        for v in range(n):
            seen, x = [], v
            while x >= 0 and x not in seen and len(seen) <= n:
                seen.append(x)
                x = tgt[x]
            if x >= 0:
                cyc = seen[seen.index(x):]
                assert len(cyc) == 2, cyc
        for v in rng.permutation(n)[: n // 6]:
            if mate[v] < 0 and tgt[v] >= 0 and mate[tgt[v]] < 0:
                mate[v], mate[tgt[v]] = tgt[v], v


def _small_components(seed):
    # components of at most 16 nodes: no node has more than 15 neighbours at
    # any level, so K = 16 lists hold every valid neighbour
    rng = np.random.default_rng(seed)
    sizes = rng.integers(3, 17, size=60).tolist()
    return inputs.planted_components(sizes, 9, 4, seed=seed)


def test_constant_model_is_plain_priority():
    # mutual lists are the whole valid neighbourhoods and (const, eta, id)
    # orders as (eta, id)
    g = _small_components(11)
    omega, delta, K, pi = 6, 30, 16, 4
    size, candK, csK = _level(g, omega, delta, K)
    assert (candK[:, -1] < 0).all()
    _, _, cand, cs = oracle.learned_level(g, size, omega, delta, 0, candK.ravel(), csK.ravel(), pi,
                                          inputs.constant_merge_model(7))
    plain_c, plain_s = oracle.propose(g, size, omega, delta, pi=pi)
    assert np.array_equal(cand.reshape(-1, pi), plain_c)
    assert np.array_equal(cs.reshape(-1, pi), plain_s)


@pytest.mark.parametrize("seed,omega,delta", [(2, 4, 12), (3, 8, 40), (4, 16, 64)])
def test_constant_model_partition_is_plain_partition(seed, omega, delta):
    g = _small_components(seed)
    plain = oracle.partition(g, omega, delta, seed=1, trace=True)
    lrn = oracle.partition(g, omega, delta, seed=1, trace=True, learned_k=16, model=inputs.constant_merge_model(-3))
    assert plain.status == lrn.status == oracle.OK
    assert np.array_equal(plain.part, lrn.part)
    assert plain.stats == lrn.stats and plain.trace == lrn.trace
    assert plain.stats["levels"] > 2


def test_learned_partition_valid_and_deterministic():
    g = inputs.random_snn(1500, 15, seed=3)
    a = oracle.partition(g, 32, 160, seed=0, learned_k=16, model=inputs.random_merge_model(1))
    b = oracle.partition(g, 32, 160, seed=0, learned_k=16, model=inputs.random_merge_model(1))
    c = oracle.partition(g, 32, 160, seed=0, learned_k=16, model=inputs.random_merge_model(2))
    assert a.status == oracle.OK and a.stats["violations"] == 0
    assert np.array_equal(a.part, b.part)
    assert c.status == oracle.OK and c.stats["violations"] == 0
    assert not np.array_equal(a.part, c.part)


def test_learned_options_checked():
    g = inputs.random_snn(100, 4, seed=0)
    assert oracle.partition(g, 8, 40, learned_k=16).status == oracle.ERR_INVALID_ARG   # no model
    assert oracle.partition(g, 8, 40, learned_k=3, model=zero_model()).status == oracle.ERR_INVALID_ARG   # K < Pi
    assert oracle.partition(g, 8, 40, learned_k=17, model=zero_model()).status == oracle.ERR_INVALID_ARG


def test_hand_derived_example():
    """tests/golden/learned_small.json: features, scores and C(n) of a 5-node
    level, each derived by hand (the derivation is in the file)."""
    import json
    import os
    d = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "learned_small.json")))
    g = inputs.Hypergraph(num_nodes=d["num_nodes"], offsets=np.array(d["offsets"], np.int32),
                          pins=np.array(d["pins"], np.int32))
    size = np.ones(d["num_nodes"], np.int32)
    K, pi = d["K"], d["pi"]
    candK, csK = oracle.propose(g, size, d["omega"], d["delta"], seed=0, level=d["level"], pi=K,
                                permille=d["permille"])
    assert candK.tolist() == d["cand_K"]
    m = inputs.constant_merge_model(0)
    m.b1[0], m.w1[0, 0], m.w2[0, 0], m.w3[0] = (d["model"][k] for k in ("b1_0", "w1_0_0", "w2_0_0", "w3_0"))
    feat, rank, cand, cs = oracle.learned_level(g, size, d["omega"], d["delta"], d["level"], candK.ravel(),
                                                csK.ravel(), pi, m)
    s = oracle.mlp_scores(feat, m)
    for v in range(d["num_nodes"]):
        for j in range(K):
            u = candK[v, j]
            if u < 0:
                continue
            assert rank[v * K + j] >= 0
            assert feat[v * K + j].tolist() == d["features"][f"{v},{u}"], (v, u)
            assert s[v * K + j] == d["scores"][f"{v},{u}"], (v, u)
    assert cand.reshape(-1, pi).tolist() == d["C"]
    assert cs.reshape(-1, pi).tolist() == d["C_eta"]


@pytest.mark.parametrize("case", ["empty", "one_node", "no_hyperedges", "singletons", "two_components"])
def test_degenerate_inputs_match_plain(case):
    # with no candidate pairs at all (or only pairs that every priority ranks alike) the
    # learned priority must give the plain result
    if case == "empty":
        g = inputs.Hypergraph(num_nodes=0, offsets=np.zeros(1, np.int32), pins=np.zeros(0, np.int32))
    elif case == "one_node":
        g = inputs.Hypergraph(num_nodes=1, offsets=np.array([0, 1], np.int32), pins=np.array([0], np.int32))
    elif case == "no_hyperedges":
        g = inputs.Hypergraph(num_nodes=9, offsets=np.zeros(1, np.int32), pins=np.zeros(0, np.int32))
    elif case == "singletons":
        g = inputs.Hypergraph(num_nodes=6, offsets=np.arange(7, dtype=np.int32), pins=np.arange(6, dtype=np.int32))
    else:   # two disjoint pairs: each node has exactly one valid neighbour
        g = inputs.Hypergraph(num_nodes=4, offsets=np.array([0, 2, 4], np.int32), pins=np.array([0, 1, 2, 3], np.int32))
    plain = oracle.partition(g, 2, 8, seed=3, trace=True)
    lrn = oracle.partition(g, 2, 8, seed=3, trace=True, learned_k=4, model=inputs.random_merge_model(1))
    assert plain.status == lrn.status == oracle.OK
    assert np.array_equal(plain.part, lrn.part) and plain.stats == lrn.stats


@pytest.mark.parametrize("k", [1, 2, 3])
def test_learned_levels_limit_the_learned_ranking_to_the_first_levels(k):
    """learned_levels = k: the first k levels are those of the fully learned
    run (a level depends only on the levels before it); the deeper levels are
    those a plain proposal makes of the hierarchy it receives."""
    g = inputs.random_snn(600, 15, seed=11)
    full = oracle.partition(g, 24, 96, seed=0, trace=True, learned_k=16, model=inputs.random_merge_model(3))
    part = oracle.partition(g, 24, 96, seed=0, trace=True, learned_k=16, model=inputs.random_merge_model(3),
                            learned_levels=k)
    assert full.status == part.status == oracle.OK
    nlev = min(k, len(full.trace) - 1)
    for lv in range(nlev):
        for key in ("n", "pins", "pairs", "iso_pairs", "valid", "iso_list", "targets_r1", "max_indeg_r1", "pairs_r1"):
            assert part.trace[lv][key] == full.trace[lv][key], (k, lv, key)
    assert part.trace[nlev]["n"] == full.trace[nlev]["n"]
    assert part.stats["violations"] == 0
    # a limit beyond the level count is the fully learned run
    same = oracle.partition(g, 24, 96, seed=0, learned_k=16, model=inputs.random_merge_model(3), learned_levels=500)
    assert np.array_equal(same.part, full.part)
    # without learned_k the limit changes nothing
    plain = oracle.partition(g, 24, 96, seed=0)
    p2 = oracle.partition(g, 24, 96, seed=0, learned_levels=1)
    assert np.array_equal(plain.part, p2.part)
    assert oracle.partition(g, 24, 96, learned_levels=-1).status == oracle.ERR_INVALID_ARG
