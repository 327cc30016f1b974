"""Seeded synthetic hypergraphs (inputs only; none of the partitioner's arithmetic).

Every generator draws from numpy's PCG64 (``numpy.random.default_rng``), whose
output is identical on x86-64 and aarch64, so the same seed gives the same
hypergraph on the build host and on the GPU host.  Hypergraphs are plain
int32 CSR: ``offsets[E+1]``, ``pins[offsets[E]]``; each hyperedge lists its
source pins first (``src_counts[e]`` of them; ``None`` means exactly one, the
first pin), then its destinations in ascending id order.

The shapes follow the spiking-network workloads of the paper's Table I
(random "-rand" nets and regular layered "-model" nets):

* :func:`random_snn` -- every node owns one hyperedge: itself plus ``k``
  distinct uniform-random targets (4,096 x 31 and 16,384 x 127 workloads).
* :func:`layered_snn` -- ``layers`` grids of ``h x w x ch`` neurons; a neuron
  of every layer but the last owns a hyperedge to all channels of the 3x3
  window (border-clipped) around its position in the next layer
  (8 x 32 x 32 x 32 = 262,144 nodes, ~63.6M pins).
* :func:`random_hypergraph` -- small irregular hypergraphs for tests
  (optional multi-source hyperedges, weights, isolated nodes).

:class:`MergeModel` holds the integer parameters of the learned merge
priority (16 -> 64 -> 64 -> 1); :func:`random_merge_model` draws seeded ones.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Hypergraph:
    num_nodes: int
    offsets: np.ndarray            # int32 [E+1]
    pins: np.ndarray               # int32 [offsets[-1]]
    src_counts: np.ndarray | None = None   # int32 [E] or None (one source each)
    weights: np.ndarray | None = None      # int32 [E] or None (unit weights)
    name: str = ""

    @property
    def num_hedges(self) -> int:
        return len(self.offsets) - 1

    @property
    def num_pins(self) -> int:
        return int(self.offsets[-1])

    def edges(self):
        """Yields (src list, dst list) per hyperedge (for small test graphs)."""
        for e in range(self.num_hedges):
            seg = self.pins[self.offsets[e]:self.offsets[e + 1]].tolist()
            k = 1 if self.src_counts is None else int(self.src_counts[e])
            yield seg[:k], seg[k:]


def _csr(rows, n, name="", src_counts=None, weights=None) -> Hypergraph:
    sizes = np.fromiter((len(r) for r in rows), dtype=np.int64, count=len(rows))
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    pins = np.concatenate([np.asarray(r, dtype=np.int32) for r in rows]) if rows else np.zeros(0, np.int32)
    return Hypergraph(n, off.astype(np.int32), pins.astype(np.int32), src_counts, weights, name)


_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) of counters x
    (uint64 arrays, wrapping arithmetic): the same stream on every machine
    and numpy version."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def random_snn(n: int, k: int, seed: int = 0) -> Hypergraph:
    """Node i owns hyperedge {i} + k distinct uniform targets != i (sorted).

    Target candidates of node i are splitmix64(counter(seed, i, j)) mod
    (n - 1), shifted past i, for j = 0, 1, ...; the first k distinct ones
    are kept."""
    assert n >= 2 and k <= n - 1 and n < (1 << 28)
    pins = np.empty((n, k + 1), dtype=np.int32)
    pins[:, 0] = np.arange(n, dtype=np.int32)
    draw = 2 * k + 16
    base = np.uint64(seed & 0xFFFF) << np.uint64(48)
    for i in range(n):
        got = np.empty(0, dtype=np.int64)
        j0 = 0
        while got.size < k:
            j = np.arange(j0, j0 + draw, dtype=np.uint64)
            c = (splitmix64(base | (np.uint64(i) << np.uint64(20)) | j) % np.uint64(n - 1)).astype(np.int64)
            c = c + (c >= i)          # skip the source itself
            allc = np.concatenate([got, c])
            _, first = np.unique(allc, return_index=True)
            got = allc[np.sort(first)][:k]
            j0 += draw
        pins[i, 1:] = np.sort(got)
    off = np.arange(0, n * (k + 1) + 1, k + 1, dtype=np.int64)
    return Hypergraph(n, off.astype(np.int32), pins.reshape(-1), None, None, f"random_snn_{n}x{k}")


def _uniform01(x: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64(x)."""
    return (splitmix64(x) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def powerlaw_snn(n: int, seed: int, alpha: float = 2.2, smin: int = 2, smax: int = 1024) -> Hypergraph:
    """Node i owns hyperedge {i} + (s_i - 1) distinct uniform targets != i,
    s_i from the discrete power law P(s) ~ s^-alpha on [smin, min(smax, n)]
    (inverse CDF), targets from a SplitMix64 counter stream; pins sorted."""
    hi = min(smax, n)
    sv = np.arange(smin, hi + 1, dtype=np.float64)
    cdf = np.cumsum(sv ** -alpha)
    cdf /= cdf[-1]
    base = np.uint64(seed & 0xFFFF) << np.uint64(48)
    u = _uniform01(base | np.arange(n, dtype=np.uint64))
    sizes = (smin + np.searchsorted(cdf, u, side="right")).astype(np.int64)
    sizes = np.minimum(sizes, hi)
    need = sizes - 1
    # candidates in rounds: 2 * need + 8 draws per hyperedge, then more for
    # the hyperedges still short of distinct targets; first occurrences kept
    tgt_c = np.empty(0, dtype=np.int64)
    tgt_e = np.empty(0, dtype=np.int64)
    tgt_j = np.empty(0, dtype=np.int64)
    draws = 2 * need + 8
    done = np.zeros(n, dtype=np.int64)   # draws used so far per hyperedge
    got = np.zeros(n, dtype=np.int64)
    while True:
        todo = np.nonzero(got < need)[0]
        if todo.size == 0:
            break
        cnt = draws[todo]
        e_idx = np.repeat(todo, cnt)
        j = np.repeat(done[todo], cnt) + np.arange(cnt.sum(), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        ctr = base | (np.uint64(1) << np.uint64(47)) | (e_idx.astype(np.uint64) << np.uint64(24)) | j.astype(np.uint64)
        c = (splitmix64(ctr) % np.uint64(max(n - 1, 1))).astype(np.int64)
        c = c + (c >= e_idx)
        done[todo] += cnt
        draws[todo] *= 2
        c = np.concatenate([tgt_c, c])
        e_idx = np.concatenate([tgt_e, e_idx])
        j = np.concatenate([tgt_j, j])
        order = np.lexsort((j, c, e_idx))
        c, e_idx, j = c[order], e_idx[order], j[order]
        first = np.ones(c.size, dtype=bool)
        first[1:] = (c[1:] != c[:-1]) | (e_idx[1:] != e_idx[:-1])
        c, e_idx, j = c[first], e_idx[first], j[first]
        order = np.lexsort((j, e_idx))
        c, e_idx, j = c[order], e_idx[order], j[order]
        start = np.searchsorted(e_idx, np.arange(n))
        rank = np.arange(c.size) - start[e_idx]
        keep = rank < need[e_idx]
        tgt_c, tgt_e, tgt_j = c[keep], e_idx[keep], j[keep]
        got = np.bincount(tgt_e, minlength=n)
    order = np.lexsort((tgt_c, tgt_e))
    tgt = tgt_c[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    pins = np.empty(int(off[-1]), dtype=np.int32)
    pins[off[:-1]] = np.arange(n, dtype=np.int32)
    mask = np.ones(pins.size, dtype=bool)
    mask[off[:-1]] = False
    pins[mask] = tgt.astype(np.int32)
    return Hypergraph(n, off.astype(np.int32), pins, None, None, f"powerlaw_snn_{n}_{seed}")


def batch_snn(count: int, seed: int = 0, n_min: int = 1000, n_max: int = 64000):
    """Independent instances: n log-uniform in [n_min, n_max], power-law
    hyperedge sizes (powerlaw_snn), Omega uniform in {2^8..2^12}, Delta =
    4 Omega.  Returns [(Hypergraph, Omega, Delta, partition seed)]."""
    base = (np.uint64(seed & 0xFFFF) << np.uint64(48)) | (np.uint64(1) << np.uint64(46))
    u = _uniform01(base | np.arange(2 * count, dtype=np.uint64))
    out = []
    for i in range(count):
        n = int(np.exp(np.log(n_min) + u[2 * i] * (np.log(n_max) - np.log(n_min))))
        om = 1 << (8 + min(int(u[2 * i + 1] * 5), 4))
        out.append((powerlaw_snn(n, (seed * 7919 + i) & 0xFFFF), om, 4 * om, i))
    return out


def layered_snn(layers: int = 8, h: int = 32, w: int = 32, ch: int = 32) -> Hypergraph:
    """Locally connected layered net; node id = ((L*h + y)*w + x)*ch + c."""
    n = layers * h * w * ch
    rows_sizes = []
    pin_blocks = []
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    for L in range(layers - 1):
        base_next = (L + 1) * h * w * ch
        for y in range(h):
            y0, y1 = max(0, y - 1), min(h, y + 2)
            for x in range(w):
                x0, x1 = max(0, x - 1), min(w, x + 2)
                tgt = ((base_next + (ys[y0:y1, x0:x1] * w + xs[y0:y1, x0:x1]) * ch)[..., None]
                       + np.arange(ch)[None, None, :]).reshape(-1)
                src = ((L * h + y) * w + x) * ch + np.arange(ch)
                blk = np.empty((ch, 1 + tgt.size), dtype=np.int32)
                blk[:, 0] = src
                blk[:, 1:] = tgt[None, :]
                pin_blocks.append(blk.reshape(-1))
                rows_sizes.append(np.full(ch, 1 + tgt.size, dtype=np.int64))
    sizes = np.concatenate(rows_sizes)
    off = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    pins = np.concatenate(pin_blocks)
    return Hypergraph(n, off.astype(np.int32), pins, None, None, f"layered_snn_{layers}x{h}x{w}x{ch}")


def random_hypergraph(n: int, e: int, max_size: int, seed: int = 0, multi_src: bool = False,
                      weights: bool = False, isolated: int = 0, max_weight: int = 5) -> Hypergraph:
    """Small irregular hypergraph: e hyperedges of 1..max_size distinct pins
    over the first n - isolated nodes (the last ``isolated`` nodes touch none)."""
    rng = np.random.default_rng(seed)
    live = max(n - isolated, 1)
    rows, src = [], []
    for _ in range(e):
        s = int(rng.integers(1, min(max_size, live) + 1))
        pins = rng.choice(live, size=s, replace=False).astype(np.int32)
        k = int(rng.integers(0, s + 1)) if multi_src else 1
        head, tail = np.sort(pins[:k]), np.sort(pins[k:])
        rows.append(np.concatenate([head, tail]))
        src.append(k)
    g = _csr(rows, n, f"random_hg_{n}_{e}_{seed}",
             np.asarray(src, dtype=np.int32) if multi_src else None,
             rng.integers(1, max_weight + 1, size=e).astype(np.int32) if weights else None)
    return g


def planted_components(sizes, edges_per_comp: int, edge_size: int, seed: int = 0) -> Hypergraph:
    """Disjoint components (node blocks of the given sizes); every hyperedge
    stays inside one component."""
    rng = np.random.default_rng(seed)
    rows = []
    base = 0
    for s in sizes:
        for _ in range(edges_per_comp):
            k = min(edge_size, s)
            rows.append(np.sort(base + rng.choice(s, size=k, replace=False)).astype(np.int32))
        base += s
    perm = rng.permutation(len(rows))
    rows = [rows[i] for i in perm]
    return _csr(rows, int(sum(sizes)), "planted")


def workload(name: str, seed: int = 0) -> Hypergraph:
    """Named workloads used by the benchmark and the parity tests."""
    if name == "random_snn_4k":
        return random_snn(4096, 31, seed)
    if name == "random_snn_16k":
        return random_snn(16384, 127, seed)
    if name == "layered_snn_262k":
        return layered_snn(8, 32, 32, 32)
    if name == "layered_snn_16k":
        return layered_snn(4, 16, 16, 16)
    if name == "layered_snn_65k":
        return layered_snn(8, 16, 16, 32)
    raise KeyError(name)


# Omega, Delta of each named workload (paper Table I: 2^10/2^12 for the random
# nets, 2^12/2^16 for the layered nets; 256/1024 for the small random net)
CONSTRAINTS = {
    "random_snn_4k": (256, 1024),
    "random_snn_16k": (1 << 10, 1 << 12),
    "layered_snn_262k": (1 << 12, 1 << 16),
    "layered_snn_16k": (1 << 10, 1 << 14),
    "layered_snn_65k": (1 << 12, 1 << 16),
}


@dataclass
class MergeModel:
    """Parameters of the learned merge priority: weight codes in [-127, 127],
    biases with |b| <= 2^30, right shifts 0..30 after the two hidden layers."""
    w1: np.ndarray   # int8 [64, 16]
    w2: np.ndarray   # int8 [64, 64]
    w3: np.ndarray   # int8 [64]
    b1: np.ndarray   # int32 [64]
    b2: np.ndarray   # int32 [64]
    b3: int
    shift1: int
    shift2: int


def random_merge_model(seed: int, bias_scale: int = 2048, shift1: int = 6, shift2: int = 8,
                       wmax: int = 127) -> MergeModel:
    """Uniform weight codes in [-wmax, wmax] and biases in
    [-bias_scale, bias_scale]; the default shifts keep most hidden codes
    inside 0..255 for features of the usual magnitude."""
    r = np.random.default_rng(seed)
    return MergeModel(
        w1=r.integers(-wmax, wmax + 1, size=(64, 16)).astype(np.int8),
        w2=r.integers(-wmax, wmax + 1, size=(64, 64)).astype(np.int8),
        w3=r.integers(-wmax, wmax + 1, size=64).astype(np.int8),
        b1=r.integers(-bias_scale, bias_scale + 1, size=64).astype(np.int32),
        b2=r.integers(-bias_scale, bias_scale + 1, size=64).astype(np.int32),
        b3=int(r.integers(-bias_scale, bias_scale + 1)),
        shift1=shift1, shift2=shift2)


def constant_merge_model(b3: int = 7) -> MergeModel:
    """All weights zero: every pair scores b3."""
    return MergeModel(w1=np.zeros((64, 16), np.int8), w2=np.zeros((64, 64), np.int8), w3=np.zeros(64, np.int8),
                      b1=np.zeros(64, np.int32), b2=np.zeros(64, np.int32), b3=b3, shift1=0, shift2=0)
