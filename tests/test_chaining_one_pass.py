"""The CUDA path's one-pass chaining round, checked on the CPU against the
oracle's chaining (Sec. VI-C).

The oracle runs each chaining round as the paper describes it: every free
chain end chooses, then each chosen move takes its best chooser, then the
links are made.  The cluster sequencing kernel fuses a round's links into the
next round's pass: a chooser finds out from the slot of the move it chose
whether it won; a move counts as taken when it has a predecessor or a key in
the previous round's slots; slots rotate over three arrays.  This test restates
that one-pass form in Python and checks that it yields the oracle's sequence
on random move sets, and that a one-pass round which forgets the previous
round's slots does not.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import inputs


def one_pass_sequence(node, src, dst, gain, size, nin, nparts, window, rounds, use_prev_slots=True):
    M = len(node)
    first = np.zeros(nparts + 1, dtype=np.int64)
    for p in src:
        first[p + 1] += 1
    first = np.cumsum(first)
    pred = [-1] * M
    pred_before = [-1] * M   # predecessors written in earlier passes (what a pass may read)
    succ = [-1] * M
    choice = [-1] * M
    pen = [0] * M
    slots = [dict(), dict(), dict()]   # acc[r % 3]: move -> best (-penalty, chooser node)
    linked = [False] * (rounds + 1)

    def key(i):
        return (-pen[i], node[i])

    last = -1
    for r in range(rounds):
        if r > 0 and not linked[r - 1]:
            break
        prev, cur = slots[(r + 2) % 3], slots[r % 3]
        slots[(r + 1) % 3] = dict()
        new_choice, new_pen = [-1] * M, [0] * M
        for i in range(M):
            end_taken = succ[i] >= 0
            if r > 0 and choice[i] >= 0 and prev.get(choice[i]) == key(i):
                pred[choice[i]] = i   # (in the kernel, written during this same pass)
                succ[i] = choice[i]
                end_taken = True
            if end_taken:
                continue
            d = dst[i]
            seen, best, bG, bpen = 0, -1, None, 0
            for j in range(first[d], first[d + 1]):
                if seen >= window:
                    break
                taken = pred_before[j] >= 0 or (use_prev_slots and r > 0 and j in prev)
                if taken or j == i:
                    continue
                seen += 1
                p = 10 * abs(int(size[node[i]]) - int(size[node[j]])) + abs(int(nin[node[i]]) - int(nin[node[j]]))
                G = int(gain[j]) * 10_000_000 - p
                if best < 0 or G > bG:
                    best, bG, bpen = j, G, p
            new_choice[i], new_pen[i] = best, bpen
            if best >= 0:
                k = (-bpen, node[i])
                if best not in cur or k > cur[best]:
                    cur[best] = k
                linked[r] = True
        choice, pen = new_choice, new_pen
        last = r
        pred_before = list(pred)
    if last >= 0 and linked[last] and last == rounds - 1:
        cur = slots[last % 3]
        for i in range(M):
            if choice[i] >= 0 and cur.get(choice[i]) == key(i):
                pred[choice[i]] = i
                succ[i] = choice[i]
    # chains (paths from their heads, cycles from their smallest node), by (gain desc, head node asc)
    # (a variant whose links are not a set of paths and cycles returns None)
    chains, vis = [], [False] * M
    for i in range(M):
        if pred[i] < 0:
            c, j = [], i
            while j >= 0:
                if vis[j]:
                    return None
                vis[j] = True
                c.append(j)
                j = succ[j]
            chains.append(c)
    for i in range(M):
        if not vis[i]:
            c, j = [], i
            while True:
                if vis[j] or j < 0:
                    return None
                vis[j] = True
                c.append(j)
                j = succ[j]
                if j == i:
                    break
            h = min(range(len(c)), key=lambda t: node[c[t]])
            chains.append(c[h:] + c[:h])
    chains.sort(key=lambda c: (-sum(int(gain[j]) for j in c), node[c[0]]))
    return [j for c in chains for j in c]


def random_moves(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(30, 90))
    g = inputs.random_hypergraph(n, 3 * n, 6, seed=seed, multi_src=True)
    nparts = int(rng.integers(3, 9))
    M = int(rng.integers(10, n))
    node = rng.choice(n, size=M, replace=False).astype(np.int32)
    src = rng.integers(0, nparts, size=M).astype(np.int32)
    dst = ((src + rng.integers(1, nparts, size=M)) % nparts).astype(np.int32)
    gain = rng.integers(1, 4, size=M).astype(np.int64)
    order = np.lexsort((node, -gain, src))
    node, src, dst, gain = node[order], src[order], dst[order], gain[order]
    size = rng.integers(1, 4, size=n).astype(np.int32)
    nin = np.zeros(n, dtype=np.int64)
    k = g.src_counts
    for e in range(g.num_hedges):
        for j in range(g.offsets[e] + k[e], g.offsets[e + 1]):
            nin[g.pins[j]] += 1
    return g, size, nin, nparts, node, src, dst, gain


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("window,rounds", [(256, 16), (2, 16), (3, 2)])
def test_one_pass_rounds_give_the_oracle_sequence(seed, window, rounds):
    g, size, nin, nparts, node, src, dst, gain = random_moves(seed)
    want = oracle.sequence(g, size, nparts, node, src, dst, gain, window=window, rounds=rounds).tolist()
    got = one_pass_sequence(node.tolist(), src, dst, gain, size, nin, nparts, window, rounds)
    assert got == want


def test_forgetting_the_previous_slots_is_caught():
    differs = 0
    for seed in range(12):
        g, size, nin, nparts, node, src, dst, gain = random_moves(seed)
        want = oracle.sequence(g, size, nparts, node, src, dst, gain).tolist()
        got = one_pass_sequence(node.tolist(), src, dst, gain, size, nin, nparts, 256, 16, use_prev_slots=False)
        differs += got != want
    assert differs > 0
