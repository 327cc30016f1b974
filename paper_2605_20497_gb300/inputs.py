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
* :func:`gaussian_layered_snn` -- a large sparse layered network: 16 grids
  of 512 x 512 neurons; hyperedge sizes geometric (mean 84, cap 1024),
  targets Gaussian-local (sigma = 4 cells) in the next layer.
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


def _popcount64(x: np.ndarray) -> np.ndarray:
    """Set bits of each uint64 (SWAR bit counting, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        x = x - ((x >> np.uint64(1)) & np.uint64(0x5555555555555555))
        x = (x & np.uint64(0x3333333333333333)) + ((x >> np.uint64(2)) & np.uint64(0x3333333333333333))
        x = (x + (x >> np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
        return ((x * np.uint64(0x0101010101010101)) >> np.uint64(56)).astype(np.int64)


def _geometric_thresholds(mean: int, cap: int) -> np.ndarray:
    """P(s > k) = (1 - 1/mean)^k for k = 1 .. cap-1, each the correctly
    rounded double of the exact rational power, ascending."""
    from fractions import Fraction
    q = Fraction(mean - 1, mean)
    t, x = [], Fraction(1)
    for _ in range(1, cap):
        x *= q
        t.append(float(x))
    return np.asarray(t[::-1], dtype=np.float64)


def _gaussian_key(seed: int, stream: int, e: np.ndarray, j: np.ndarray) -> np.ndarray:
    # counter of draw j of hyperedge e in one of the streams (0 size, 1 rows, 2 columns)
    return ((np.uint64(seed & 0xFF) << np.uint64(56)) | (np.uint64(stream) << np.uint64(52))
            | (e.astype(np.uint64) << np.uint64(28)) | j.astype(np.uint64))


def gaussian_offsets(seed: int, stream: int, e: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Centred binomial B(64, 1/2) - 32 of the counters: mean 0, variance 16
    (sigma = 4 cells), support -32..32; the de Moivre-Laplace approximation of
    round(N(0, 16)) in exact integer arithmetic."""
    return _popcount64(splitmix64(_gaussian_key(seed, stream, e, j))) - 32


def _gaussian_chunk(args):
    """Pins and hyperedge sizes of hyperedges a..b-1 of gaussian_layered_snn."""
    a, b, h, w, mean, cap, seed, rounds = args
    n_layer = h * w
    thr = _geometric_thresholds(mean, cap)
    e = np.arange(a, b, dtype=np.int64)
    m = b - a
    u = _uniform01(_gaussian_key(seed, 0, e, np.zeros(m, np.int64)))
    need = (thr.size - np.searchsorted(thr, u, side="right")).astype(np.int64)   # s - 1
    lay, y, x = e // n_layer, (e // w) % h, e % w
    # accepted targets, as packed keys row << 40 | draw << 23 | target offset in the next layer
    done = []
    acc = np.zeros(0, np.uint64)
    have = np.zeros(m, np.int64)
    next_j = np.zeros(m, np.int64)
    base_t = (lay + 1) * n_layer
    M23, M17 = np.uint64((1 << 23) - 1), np.uint64((1 << 17) - 1)
    for _ in range(rounds):
        deficit = need - have
        cnt = np.where(deficit > 0, (deficit * 5 + 3) // 4 + 4, 0)
        tot = int(cnt.sum())
        if tot == 0:
            break
        rows = np.repeat(np.arange(m, dtype=np.int64), cnt)
        start = np.cumsum(cnt) - cnt
        j = next_j[rows] + (np.arange(tot, dtype=np.int64) - start[rows])
        next_j += cnt
        ty = y[rows] + gaussian_offsets(seed, 1, e[rows], j)
        tx = x[rows] + gaussian_offsets(seed, 2, e[rows], j)
        ok = (ty >= 0) & (ty < h) & (tx >= 0) & (tx < w)
        new = ((rows[ok].astype(np.uint64) << np.uint64(40)) | (j[ok].astype(np.uint64) << np.uint64(23))
               | (ty[ok] * w + tx[ok]).astype(np.uint64))
        # rows still short of targets: their accepted and new draws, first draw of each target
        allk = np.concatenate([acc, new])
        rt = ((allk >> np.uint64(40)) << np.uint64(23)) | (allk & M23)   # row, target
        srt = np.lexsort(((allk >> np.uint64(23)) & M17, rt))
        rt_s = rt[srt]
        first = np.ones(rt_s.size, bool)
        first[1:] = rt_s[1:] != rt_s[:-1]
        allk = np.sort(allk[srt[first]])                                # by row, then draw
        r_all = (allk >> np.uint64(40)).astype(np.int64)
        cnt_r = np.bincount(r_all, minlength=m)
        rank = np.arange(r_all.size) - (np.cumsum(cnt_r) - cnt_r)[r_all]
        allk = allk[rank < need[r_all]]
        r_all = (allk >> np.uint64(40)).astype(np.int64)
        have = np.where(deficit > 0, np.bincount(r_all, minlength=m), have)   # rows done earlier keep theirs
        full = have[r_all] == need[r_all]
        done.append(allk[full])                                          # complete rows leave the loop
        acc = allk[~full]
    done.append(acc)
    allk = np.concatenate(done)
    acc_r = (allk >> np.uint64(40)).astype(np.int64)
    acc_t = base_t[acc_r] + (allk & M23).astype(np.int64)
    srt = np.lexsort((acc_t, acc_r))
    acc_r, acc_t = acc_r[srt], acc_t[srt]
    size = 1 + have
    off = np.cumsum(size) - size
    out = np.empty(int(size.sum()), dtype=np.int32)
    out[off] = e
    rank = np.arange(acc_r.size) - (np.cumsum(have) - have)[acc_r]
    out[off[acc_r] + 1 + rank] = acc_t
    return out, size


def gaussian_layered_snn(layers: int = 16, h: int = 512, w: int = 512, mean: int = 84, cap: int = 1024,
                         seed: int = 0, rounds: int = 8, chunk: int = 1 << 16, workers: int = 1) -> Hypergraph:
    """Large sparse layered network: every node of layers 0..layers-2 owns a
    hyperedge {itself} + (s - 1) distinct targets in the next layer.  s is
    geometric with the given mean, capped at `cap` (P(s > k) = (1-1/mean)^k).
    A target lies at (y + dy, x + dx) in the next layer, with dy, dx drawn
    from gaussian_offsets (sigma = 4 cells); draws that leave the grid or
    repeat a target are drawn again.  Redrawing is bounded: `rounds` rounds,
    each drawing 1.25 x the missing targets + 4; a hyperedge that still lacks
    targets (only nodes near a border with large s) keeps those it has.
    Targets are sorted ascending after the source.  Chunks of `chunk`
    hyperedges are independent; `workers` > 1 generates them in a process
    pool (started with spawn) with the same result."""
    n_layer = h * w
    n, E = layers * n_layer, (layers - 1) * n_layer
    assert E < (1 << 24) and cap <= 1024 and h <= 1 << 16 and w <= 1 << 16
    jobs = [(a, min(E, a + chunk), h, w, mean, cap, seed, rounds) for a in range(0, E, chunk)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            res = list(ex.map(_gaussian_chunk, jobs))
    else:
        res = [_gaussian_chunk(j) for j in jobs]
    offs = np.zeros(E + 1, dtype=np.int64)
    np.cumsum(np.concatenate([r[1] for r in res]) if res else np.zeros(0, np.int64), out=offs[1:])
    assert offs[-1] < (1 << 31)
    pins = np.concatenate([r[0] for r in res]) if res else np.zeros(0, np.int32)
    return Hypergraph(n, offs.astype(np.int32), pins, None, None, f"gaussian_layered_snn_{layers}x{h}x{w}")


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
    if name == "gaussian_layered_snn_4m":
        import os
        return gaussian_layered_snn(16, 512, 512, 84, 1024, seed, workers=min(16, os.cpu_count() or 1))
    if name == "gaussian_layered_snn_1m":
        # the same family on 256 x 256 grids: a quarter of the nodes and pins
        import os
        return gaussian_layered_snn(16, 256, 256, 84, 1024, seed, workers=min(16, os.cpu_count() or 1))
    raise KeyError(name)


# Omega, Delta of each named workload (paper Table I: 2^10/2^12 for the random
# nets, 2^12/2^16 for the layered nets; 256/1024 for the small random net)
CONSTRAINTS = {
    "random_snn_4k": (256, 1024),
    "random_snn_16k": (1 << 10, 1 << 12),
    "layered_snn_262k": (1 << 12, 1 << 16),
    "layered_snn_16k": (1 << 10, 1 << 14),
    "layered_snn_65k": (1 << 12, 1 << 16),
    "gaussian_layered_snn_4m": (1 << 12, 1 << 16),
    "gaussian_layered_snn_1m": (1 << 12, 1 << 16),
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
