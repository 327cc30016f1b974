"""The CUDA path's in-sequence gains and prefix validity, restated on the CPU and
checked against the oracle (Eq. 14-15, Sec. VI-D).

The oracle simulates the sequence move by move.  The CUDA path evaluates every
move at once: per hyperedge, the move at sequence rank r sees pins(p, e) = the
count before the sequence + the moves of ranks < r of pins of e into p - those
out of p (pins_in the same over destination pins), which gives its share of the
in-sequence gain and of the change of D(p_s) and D(p_d).  The validity of every
prefix then follows from per-part running sums of capacity events: each change
of a part between valid and invalid adds +1 or -1 at its move, and a prefix is
valid when the parts invalid at the start plus those changes sum to zero.
This test restates both in numpy and compares the in-sequence gains, the best
prefix and its gain with the oracle's on random partitions and move sequences.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import inputs


def by_rank(g, size, rho, nparts, node, dst, omega, delta):
    n, E = g.num_nodes, g.num_hedges
    nsrc = g.src_counts if g.src_counts is not None else np.ones(E, dtype=np.int32)
    w = g.weights if g.weights is not None else np.ones(E, dtype=np.int32)
    M = len(node)
    rank = np.full(n, -1)
    rank[node] = np.arange(M)
    src = rho[node]
    gseq = np.zeros(M, dtype=np.int64)
    dDs = np.zeros(M, dtype=np.int64)
    dDd = np.zeros(M, dtype=np.int64)
    D0 = np.zeros(nparts, dtype=np.int64)
    for e in range(E):
        a, b = int(g.offsets[e]), int(g.offsets[e + 1])
        pins = g.pins[a:b]
        is_dst = np.arange(b - a) >= nsrc[e]
        cnt = np.bincount(rho[pins], minlength=nparts)
        cin = np.bincount(rho[pins[is_dst]], minlength=nparts)
        D0 += cin > 0
        moved = [(int(rank[v]), j) for j, v in enumerate(pins) if rank[v] >= 0]
        for r, j in moved:
            # counts this move sees: the list's + the earlier moves of e's pins into p - out of p
            earlier = [(rr, jj) for rr, jj in moved if rr < r]
            def seen(p, dst_only):
                c = (cin if dst_only else cnt)[p]
                for rr, jj in earlier:
                    if dst_only and not is_dst[jj]:
                        continue
                    c += int(dst[rr] == p) - int(src[rr] == p)
                return c
            ps, pd = int(src[r]), int(dst[r])
            gseq[r] += int(w[e]) * (int(seen(ps, False) == 1) - int(seen(pd, False) == 0))
            if is_dst[j]:
                dDs[r] -= int(seen(ps, True) == 1)
                dDd[r] += int(seen(pd, True) == 0)
    # validity of every prefix from per-part running sums of capacity events
    psize = np.bincount(rho, weights=size, minlength=nparts).astype(np.int64)
    bad0 = int(np.sum((psize > omega) | (D0 > delta)))
    viol = np.zeros(M, dtype=np.int64)
    run_s, run_d = psize.copy(), D0.copy()
    for r in range(M):   # events in sequence order; per part only its own events change its sums
        for p, ds, dd in ((src[r], -size[node[r]], dDs[r]), (dst[r], size[node[r]], dDd[r])):
            before = run_s[p] > omega or run_d[p] > delta
            run_s[p] += ds
            run_d[p] += dd
            after = run_s[p] > omega or run_d[p] > delta
            viol[r] += int(after) - int(before)
    cum = np.cumsum(gseq)
    nbad = bad0 + np.cumsum(viol)
    best, bestk = 0, 0
    for k in range(M):
        if nbad[k] == 0 and cum[k] >= best:
            best, bestk = int(cum[k]), k + 1
    return gseq, (bestk if best > 0 else 0), best


@pytest.mark.parametrize("seed", range(10))
def test_rank_evaluation_matches_the_oracle(seed):
    rng = np.random.default_rng(500 + seed)
    g = inputs.random_hypergraph(50, 80, 8, seed=seed, multi_src=seed % 2 == 0, weights=seed % 3 == 0)
    n = g.num_nodes
    nparts = int(rng.integers(3, 7))
    rho = rng.integers(0, nparts, n).astype(np.int32)
    size = rng.integers(1, 4, n).astype(np.int32)
    node = rng.permutation(n)[: int(rng.integers(5, 30))].astype(np.int32)
    dst = np.array([(rho[v] + rng.integers(1, nparts)) % nparts for v in node], np.int32)
    psize = np.bincount(rho, weights=size, minlength=nparts)
    omega = int(psize.max()) + int(rng.integers(0, 3))
    delta = int(rng.integers(20, 60))
    want = oracle.inseq_and_prefix(g, size, rho, nparts, node, dst, omega, delta)
    gseq, k, bg = by_rank(g, size, rho, nparts, node, dst, omega, delta)
    assert np.array_equal(gseq, want[0])
    assert (k, bg) == (want[1], want[2])


def test_counting_source_pins_toward_inbound_is_caught():
    """Letting moved source pins change pins_in (they are not inbound) breaks
    the equality on some case, so the check above can tell."""
    import inspect
    src_code = inspect.getsource(by_rank).replace("if dst_only and not is_dst[jj]:", "if False:")
    ns = {}
    exec(src_code, {"np": np}, ns)
    wrong = ns["by_rank"]
    differs = 0
    for seed in range(10):
        rng = np.random.default_rng(500 + seed)
        g = inputs.random_hypergraph(50, 80, 8, seed=seed, multi_src=True)
        n = g.num_nodes
        nparts = int(rng.integers(3, 7))
        rho = rng.integers(0, nparts, n).astype(np.int32)
        size = rng.integers(1, 4, n).astype(np.int32)
        node = rng.permutation(n)[:25].astype(np.int32)
        dst = np.array([(rho[v] + rng.integers(1, nparts)) % nparts for v in node], np.int32)
        omega = int(np.bincount(rho, weights=size, minlength=nparts).max())
        want = oracle.inseq_and_prefix(g, size, rho, nparts, node, dst, omega, 30)
        got = wrong(g, size, rho, nparts, node, dst, omega, 30)
        differs += (got[1], got[2]) != (want[1], want[2])
    assert differs > 0
