"""The coarse incidence lists that the CUDA contraction writes by rank (no sort),
checked on the CPU against the oracle's contraction (Sec. V-E).

The CUDA path does not rebuild the coarse incidence from the coarse pins.  For
a coarse node c = {u, w} it keeps each incidence entry (v, e) of u and w by the
pin keep rule seen from the node's side, and writes it at its rank: its rank
among the kept entries of its own list plus the number of kept entries of the
partner's list (same class) below it.  This test restates that construction in
numpy and compares it with the incidence lists read off the coarse hypergraph
the oracle builds from the set definition (dst' = gamma(dst(e)),
src' = gamma(src(e)) minus dst'), on random hypergraphs and matchings.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import inputs


def incidence(n, offsets, pins, nsrc):
    """Per node: (ascending inbound hyperedges, ascending outbound hyperedges)."""
    ins = [[] for _ in range(n)]
    outs = [[] for _ in range(n)]
    for e in range(len(offsets) - 1):
        a, b = int(offsets[e]), int(offsets[e + 1])
        k = int(nsrc[e])
        for j in range(a, b):
            (outs if j - a < k else ins)[int(pins[j])].append(e)
    return [sorted(x) for x in ins], [sorted(x) for x in outs]


def rank_construction(n, ins, outs, mate, gamma):
    """The coarse lists written entry by entry at their rank, as the CUDA
    contraction does."""
    def kept(v, cls, e):
        w = mate[v]
        if w < 0:
            return True
        w_dst = e in ins[w]
        if cls == 0:
            return v < w or not w_dst
        if w_dst:
            return False
        return v < w or e not in outs[w]

    nc = int(gamma.max()) + 1 if n else 0
    rep = np.full(nc, -1)
    for v in range(n):
        if mate[v] < 0 or v < mate[v]:
            rep[gamma[v]] = v
    cin = [None] * nc
    cout = [None] * nc
    for c in range(nc):
        u = int(rep[c])
        members = [u] + ([int(mate[u])] if mate[u] >= 0 else [])
        for cls, lists, dest in ((0, ins, cin), (1, outs, cout)):
            keep = {v: [e for e in lists[v] if kept(v, cls, e)] for v in members}
            size = sum(len(x) for x in keep.values())
            slot = [None] * size
            for v in members:
                other = [x for x in members if x != v]
                for r, e in enumerate(keep[v]):
                    below = sum(1 for f in keep[other[0]] if f < e) if other else 0
                    pos = r + below
                    assert slot[pos] is None, "two entries at one rank"
                    slot[pos] = e
            dest[c] = slot
    return cin, cout


def random_matching(n, rng, frac=0.6):
    mate = np.full(n, -1, dtype=np.int32)
    perm = rng.permutation(n)
    for i in range(0, int(frac * n) // 2 * 2, 2):
        a, b = int(perm[i]), int(perm[i + 1])
        mate[a], mate[b] = b, a
    return mate


@pytest.mark.parametrize("seed", range(6))
def test_coarse_incidence_by_rank_equals_the_contraction(seed):
    rng = np.random.default_rng(100 + seed)
    g = inputs.random_hypergraph(40 + 10 * seed, 60 + 15 * seed, 7, seed=seed, multi_src=seed % 2 == 1,
                                 isolated=seed % 3)
    n = g.num_nodes
    nsrc = g.src_counts if g.src_counts is not None else np.ones(g.num_hedges, dtype=np.int32)
    size = np.ones(n, dtype=np.int32)
    mate = random_matching(n, rng)
    gamma, _, coff, cpins, cnsrc = oracle.contract(g, size, mate)
    ins, outs = incidence(n, g.offsets, g.pins, nsrc)
    nc = int(gamma.max()) + 1
    want_in, want_out = incidence(nc, coff, cpins, cnsrc)
    got_in, got_out = rank_construction(n, ins, outs, mate, gamma)
    assert got_in == want_in
    assert got_out == want_out


def test_a_wrong_class_precedence_is_caught():
    """Keeping a source entry whose partner is a destination of the same
    hyperedge (the coarse node must then be a destination only) breaks the
    equality, so the check above can tell."""
    rng = np.random.default_rng(7)
    g = inputs.random_hypergraph(60, 120, 7, seed=11, multi_src=True)
    n = g.num_nodes
    mate = random_matching(n, rng, frac=1.0)
    gamma, _, coff, cpins, cnsrc = oracle.contract(g, np.ones(n, dtype=np.int32), mate)
    ins, outs = incidence(n, g.offsets, g.pins, g.src_counts)
    want_in, want_out = incidence(int(gamma.max()) + 1, coff, cpins, cnsrc)
    # the out-lists without removing in(c): (out(u) U out(w)) instead of minus in(c)
    wrong_out = []
    for c in range(len(want_out)):
        members = [v for v in range(n) if gamma[v] == c]
        wrong_out.append(sorted(set(e for v in members for e in outs[v])))
    assert wrong_out != want_out
