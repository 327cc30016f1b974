"""Pins of the oracle's move chaining (Sec. VI-C), best-effort pairing
(Sec. V-C) and noise generator, plus checks that plausible mistakes planted
in a copy of the oracle fail them.

The chaining and pairing cases are worked by hand (tests/golden/*.json, each
with its derivation); the generator is checked against the published
SplitMix64 output stream.  The planted mistakes are compiled from textual
substitutions of the oracle source (CPU only)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2605_20497_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _graph_with_inbound_counts(n, nin, src_node):
    """A hypergraph on n nodes in which node v is a destination of exactly
    nin[v] hyperedges; every hyperedge has the single source src_node."""
    rows = []
    for t in range(max(nin.values(), default=0)):
        rows.append([src_node] + sorted(v for v in nin if nin[v] > t))
    return inputs._csr(rows, n)


def _sequence_case():
    d = json.load(open(os.path.join(GOLD, "sequence_small.json")))
    mv = d["moves"]
    n = max(m["node"] for m in mv) + 1
    g = _graph_with_inbound_counts(n, {m["node"]: m["nin"] for m in mv}, 0)
    size = np.ones(n, np.int32)
    for m in mv:
        size[m["node"]] = m["size"]
    cols = {k: np.array([m[k] for m in mv]) for k in ("node", "src", "dst", "gain")}
    return d, g, size, cols


def _sequence_names():
    d, g, size, c = _sequence_case()
    seq = oracle.sequence(g, size, d["nparts"], c["node"].astype(np.int32), c["src"].astype(np.int32),
                          c["dst"].astype(np.int32), c["gain"].astype(np.int64), window=d["window"],
                          rounds=d["rounds"])
    return [d["moves"][i]["name"] for i in seq]


def test_sequence_hand_golden():
    d, _, _, c = _sequence_case()
    # the golden lists the moves in their sorted order (p_s asc, gain desc, node asc)
    keys = list(zip(c["src"].tolist(), (-c["gain"]).tolist(), c["node"].tolist()))
    assert keys == sorted(keys)
    assert _sequence_names() == d["expected_sequence"]


def _isolated_case():
    d = json.load(open(os.path.join(GOLD, "isolated_small.json")))
    nodes = d["nodes"]
    n = len(nodes)
    g = _graph_with_inbound_counts(n + 1, {v["id"]: v["nin"] for v in nodes}, n)
    size = np.ones(n + 1, np.int32)
    cand = np.full((n + 1, 4), -1, np.int32)
    mate = np.full(n + 1, -1, np.int32)
    for v in nodes:
        size[v["id"]] = v["size"]
        if not v["isolated"]:
            cand[v["id"], 0] = 9 if v["id"] != 9 else 6
        if "matched_to" in v:
            mate[v["id"]] = v["matched_to"]
    cand[n, 0] = 0   # the source-only helper node is not isolated
    return d, g, size, cand, mate


def _isolated_pairs():
    d, g, size, cand, mate0 = _isolated_case()
    k, mate = oracle.pair_isolated(g, size, d["omega"], d["delta"], cand, mate0)
    pairs = sorted(tuple(sorted((int(v), int(mate[v])))) for v in range(len(mate))
                   if mate[v] >= 0 and mate0[v] < 0 and v < mate[v])
    return k, pairs


def test_isolated_pairing_hand_golden():
    d = json.load(open(os.path.join(GOLD, "isolated_small.json")))
    k, pairs = _isolated_pairs()
    assert k == len(d["expected_pairs"])
    assert pairs == sorted(tuple(sorted(p)) for p in d["expected_pairs"])


def test_splitmix64_published_stream():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 1234567: the k-th
    # output is the finaliser of 1234567 + k * 0x9E3779B97F4A7C15
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                16408922859458223821]
    golden = 0x9E3779B97F4A7C15
    got = [oracle.splitmix64_mix((1234567 + k * golden) % 2**64) for k in range(1, 6)]
    assert got == expected


def test_pair_noise_keys_on_the_pair():
    # the noise of Sec. V-C is symmetric and depends on seed and level
    cap = 2**40
    a = oracle.pair_noise(5, 3, 10, 20, cap)
    assert a == oracle.pair_noise(5, 3, 20, 10, cap)
    assert a != oracle.pair_noise(6, 3, 10, 20, cap)
    assert a != oracle.pair_noise(5, 4, 10, 20, cap)
    assert a != oracle.pair_noise(5, 3, 10, 21, cap)


# ------------------------------------------------- planted mistakes must fail
MUTATIONS = {
    # alpha term with the wrong sign
    "alpha_sign": [("- (__int128)10 * ds - di;", "+ (__int128)10 * ds - di;")],
    # grading a successor by the chooser's own gain
    "gain_of_chooser": [("return (__int128)m->gain * 10000000", "return (__int128)n->gain * 10000000")],
    # moves skipped for having a predecessor still use up the window
    "window_counts_skipped": [("if (pred0[j] >= 0 || j == i) continue;\n                seen++;",
                               "seen++;\n                if (pred0[j] >= 0 || j == i) continue;")],
    # acceptor ties to the smaller chooser id
    "acceptor_tie": [("(cg[i] == cg[a] && mv[i].node > mv[a].node)", "(cg[i] == cg[a] && mv[i].node < mv[a].node)")],
    # chooser ties to the later sorted position
    "chooser_tie": [("if (choice[i] < 0 || G > cg[i])", "if (choice[i] < 0 || G >= cg[i])")],
    # no window limit
    "no_window": [("j < first[d + 1] && seen < window", "j < first[d + 1]")],
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_chaining_mistake_fails_the_golden(name):
    d = json.load(open(os.path.join(GOLD, "sequence_small.json")))
    assert _sequence_names() == d["expected_sequence"]
    with oracle.variant(MUTATIONS[name]):
        assert _sequence_names() != d["expected_sequence"]
    assert _sequence_names() == d["expected_sequence"]


ISO_MUTATIONS = {
    "sort_ties_by_id_desc": [("return x->id < y->id ? -1 : (x->id > y->id);",
                              "return x->id > y->id ? -1 : (x->id < y->id);")],
    "adjacent_pairs": [("int32_t a = L[i].id, b = L[k - 1 - i].id;", "int32_t a = L[2 * i].id, b = L[2 * i + 1].id;")],
    "no_delta_check": [("&& (int64_t)g->nin[a] + g->nin[b] <= delta) {", ") {")],
}


@pytest.mark.parametrize("name", sorted(ISO_MUTATIONS))
def test_planted_pairing_mistake_fails_the_golden(name):
    d = json.load(open(os.path.join(GOLD, "isolated_small.json")))
    want = sorted(tuple(sorted(p)) for p in d["expected_pairs"])
    assert _isolated_pairs()[1] == want
    with oracle.variant(ISO_MUTATIONS[name]):
        assert _isolated_pairs()[1] != want
