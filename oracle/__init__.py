"""Test infrastructure only: ctypes wrapper of the single-threaded C oracle.

The oracle (``hp_oracle.c``) is a plain CPU statement of the partitioner of
Ronzani & Silvano (constrained multilevel coarsening + refinement, Sec. III-VI)
used to check the CUDA library bit for bit.  Only ``tests/``, the smoke check
and the benchmark's CPU-baseline leg import this module; the product path does
not.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_INVALID_ARG, ERR_BAD_CSR, ERR_INFEASIBLE = 0, 1, 2, 3
COUNT_INBOUND, COUNT_INCIDENT = 0, 1
# layout of the option vector (see hp_oracle.c)
OPT_KEYS = ("pi", "theta", "chain_window", "chain_rounds", "noise_permille", "count_kind", "max_levels",
            "learned_k", "learned_levels")
DEFAULTS = dict(pi=4, theta=16, chain_window=256, chain_rounds=16, noise_permille=100, count_kind=0, max_levels=256,
                learned_k=0, learned_levels=0)
MODEL_LEN = 64 * 16 + 64 * 64 + 64 * 3 + 3   # layout of the model vector (see hp_oracle.c)
STAT_KEYS = ("connectivity", "cut_net", "num_parts", "max_part_size", "max_part_distinct",
             "violations", "levels", "moves_applied")
TRACE_KEYS = ("n", "pins", "pairs", "iso_pairs", "conn", "moves", "reps", "parts", "valid", "iso_list",
              "targets_r1", "max_indeg_r1", "pairs_r1")
TRACE_W = len(TRACE_KEYS)   # layout of a trace record (see hp_oracle.c)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


@contextlib.contextmanager
def variant(substitutions):
    """Runs the wrapper on a copy of the oracle compiled with textual
    substitutions ``[(old, new), ...]`` (each ``old`` must occur exactly once).
    Used by the tests that check that a planted mistake fails a pin."""
    global _lib
    src = open(_SRC).read()
    for old, new in substitutions:
        if src.count(old) != 1:
            raise ValueError(f"substitution target must occur once: {old!r}")
        src = src.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        c, so = os.path.join(d, "variant.c"), os.path.join(d, "libvariant.so")
        with open(c, "w") as f:
            f.write(src)
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", so, c])
        saved = lib()
        v = ctypes.CDLL(so)
        _declare(v)
        _lib = v
        try:
            yield
        finally:
            _lib = saved


P = ctypes.c_void_p
I32, I64, U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64


def _declare(L):
    L.or_partition.argtypes = [I32, I32, P, P, P, P, I32, I32, U64, P, P, P, P]
    L.or_partition.restype = ctypes.c_int
    L.or_partition_ml.argtypes = [I32, I32, P, P, P, P, I32, I32, U64, P, P, P, P, P]
    L.or_partition_ml.restype = ctypes.c_int
    L.or_mlp_scores.argtypes = [P, I64, P, P]
    L.or_mlp_scores.restype = ctypes.c_int
    L.or_learned_level.argtypes = [I32, I32, P, P, P, P, I32, I32, I32, I32, P, P, I32, P, P, P, P, P]
    L.or_learned_level.restype = ctypes.c_int
    L.or_log_code.argtypes = [U64]
    L.or_log_code.restype = I32
    L.or_node_histogram.argtypes = [I32, I32, P, P, P, P, I32, I32, P, P, P]
    L.or_node_histogram.restype = I32
    L.or_pair_noise.argtypes = [U64, I32, I32, I32, U64]
    L.or_pair_noise.restype = U64
    L.or_propose.argtypes = [I32, I32, P, P, P, P, P, I32, I32, U64, I32, I32, I32, P, P]
    L.or_propose.restype = None
    L.or_pair_isolated.argtypes = [I32, I32, P, P, P, P, I32, I32, I32, P, P]
    L.or_pair_isolated.restype = I64
    L.or_match_round.argtypes = [I32, P, P, P]
    L.or_match_round.restype = I64
    L.or_match_all.argtypes = [I32, I32, P, P, P]
    L.or_match_all.restype = I64
    L.or_contract.argtypes = [I32, I32, P, P, P, P, P, P, P, P, P, P]
    L.or_contract.restype = I32
    L.or_objective.argtypes = [I32, I32, P, P, P, P, I32, P, P]
    L.or_objective.restype = None
    L.or_propose_moves.argtypes = [I32, I32, P, P, P, P, P, P, I32, I32, I32, P, P, P, P]
    L.or_propose_moves.restype = I32
    L.or_sequence.argtypes = [I32, I32, P, P, P, P, I32, I32, P, P, P, P, I32, I32, P]
    L.or_sequence.restype = None
    L.or_inseq_and_prefix.argtypes = [I32, I32, P, P, P, P, P, P, I32, I32, P, P, I32, I32, P, P]
    L.or_inseq_and_prefix.restype = I32
    L.or_refine_rep.argtypes = [I32, I32, P, P, P, P, P, P, I32, I32, I32, I32, I32, I32]
    L.or_refine_rep.restype = I32
    L.or_splitmix64_mix.argtypes = [U64]
    L.or_splitmix64_mix.restype = U64


def _p(a):
    return None if a is None else a.ctypes.data_as(P)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Result:
    status: int
    part: np.ndarray
    stats: dict
    trace: list


def model_vector(m) -> np.ndarray:
    """The oracle's int32 vector of a MergeModel: w1, w2, w3, b1, b2, b3,
    shift1, shift2."""
    v = np.concatenate([np.asarray(m.w1, np.int32).ravel(), np.asarray(m.w2, np.int32).ravel(),
                        np.asarray(m.w3, np.int32).ravel(), np.asarray(m.b1, np.int32).ravel(),
                        np.asarray(m.b2, np.int32).ravel(), np.array([m.b3, m.shift1, m.shift2], np.int32)])
    assert v.size == MODEL_LEN
    return np.ascontiguousarray(v, dtype=np.int32)


def partition(g, omega: int, delta: int, seed: int = 0, trace: bool = False, model=None, **opts) -> Result:
    """Full multilevel partition of hypergraph ``g`` (see paper Sec. III).
    ``model``: a MergeModel, used when the option ``learned_k`` is set."""
    unknown = set(opts) - set(DEFAULTS)
    if unknown:
        raise TypeError(f"unknown oracle option(s): {sorted(unknown)}")
    o = dict(DEFAULTS)
    o.update(opts)
    optv = np.array([o[k] for k in OPT_KEYS] + [0], dtype=np.int32)
    mv = None if model is None else model_vector(model)
    off, pins = _i32(g.offsets), _i32(g.pins)
    nsrc, w = _i32(g.src_counts), _i32(g.weights)
    part = np.zeros(max(g.num_nodes, 1), dtype=np.int32)
    stats = np.zeros(16, dtype=np.int64)
    tr = np.zeros(TRACE_W * (o["max_levels"] + 1), dtype=np.int64) if trace else None
    st = lib().or_partition_ml(g.num_nodes, g.num_hedges, _p(off), _p(pins), _p(nsrc), _p(w), omega, delta,
                               ctypes.c_uint64(seed & (2**64 - 1)), _p(optv), _p(mv), _p(part), _p(stats), _p(tr))
    sd = {k: int(stats[i]) for i, k in enumerate(STAT_KEYS)}
    levels = []
    if tr is not None and st == OK:
        for l in range(sd["levels"]):
            levels.append({k: int(tr[TRACE_W * l + i]) for i, k in enumerate(TRACE_KEYS)})
    return Result(st, part[: g.num_nodes], sd, levels)


# ---- step-level entry points (one level graph), used by the pin tests ----

def node_histogram(g, v: int, permille: int = 100):
    n = g.num_nodes
    eta0 = np.zeros(max(n, 1), dtype=np.uint64)
    inter = np.zeros(max(n, 1), dtype=np.int32)
    cap = ctypes.c_uint64(0)
    k = lib().or_node_histogram(n, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)),
                                _p(_i32(g.src_counts)), _p(_i32(g.weights)), v, permille,
                                _p(eta0), _p(inter), ctypes.byref(cap))
    return k, eta0[:n], inter[:n], int(cap.value)


def splitmix64_mix(z: int) -> int:
    return int(lib().or_splitmix64_mix(ctypes.c_uint64(z & (2**64 - 1))))


def pair_noise(seed: int, level: int, a: int, b: int, cap: int) -> int:
    return int(lib().or_pair_noise(ctypes.c_uint64(seed), level, a, b, ctypes.c_uint64(cap)))


def propose(g, size, omega, delta, seed=0, level=0, pi=4, permille=100):
    n = g.num_nodes
    cand = np.zeros(max(n * pi, 1), dtype=np.int32)
    score = np.zeros(max(n * pi, 1), dtype=np.uint64)
    lib().or_propose(n, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.src_counts)),
                     _p(_i32(g.weights)), _p(_i32(size)), omega, delta, ctypes.c_uint64(seed), level, pi,
                     permille, _p(cand), _p(score))
    return cand[: n * pi].reshape(n, pi), score[: n * pi].reshape(n, pi)


def pair_isolated(g, size, omega, delta, cand, mate):
    n, pi = cand.shape
    mate = np.ascontiguousarray(mate, dtype=np.int32).copy()
    r = lib().or_pair_isolated(n, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.src_counts)),
                               _p(_i32(size)), omega, delta, pi, _p(_i32(cand.ravel())), _p(mate))
    return int(r), mate


def match_round(target, score):
    n = len(target)
    mate = np.full(max(n, 1), -1, dtype=np.int32)
    r = lib().or_match_round(n, _p(_i32(target)), _p(np.ascontiguousarray(score, dtype=np.uint64)), _p(mate))
    return int(r), mate[:n]


def match_all(cand, score, mate=None):
    n, pi = cand.shape
    mate = np.full(n, -1, dtype=np.int32) if mate is None else np.ascontiguousarray(mate, dtype=np.int32).copy()
    r = lib().or_match_all(n, pi, _p(_i32(cand.ravel())), _p(np.ascontiguousarray(score.ravel(), dtype=np.uint64)),
                           _p(mate))
    return int(r), mate


def contract(g, size, mate):
    """Returns (gamma, coarse sizes, coarse offsets, coarse pins, coarse src counts)."""
    n, e = g.num_nodes, g.num_hedges
    gamma = np.zeros(max(n, 1), dtype=np.int32)
    size_out = np.zeros(max(n, 1), dtype=np.int32)
    off_out = np.zeros(e + 1, dtype=np.int32)
    pins_out = np.zeros(max(len(g.pins), 1), dtype=np.int32)
    nsrc_out = np.zeros(max(e, 1), dtype=np.int32)
    nc = lib().or_contract(n, e, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.src_counts)), _p(_i32(size)),
                           _p(_i32(mate)), _p(gamma), _p(size_out), _p(off_out), _p(pins_out), _p(nsrc_out))
    return gamma[:n], size_out[:nc], off_out, pins_out[: off_out[-1]], nsrc_out[:e]


def objective(g, rho, nparts):
    c, cn = ctypes.c_int64(0), ctypes.c_int64(0)
    lib().or_objective(g.num_nodes, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.weights)),
                       _p(_i32(rho)), nparts, ctypes.byref(c), ctypes.byref(cn))
    return int(c.value), int(cn.value)


def propose_moves(g, size, rho, nparts, omega, second_half):
    n = g.num_nodes
    bufs = [np.zeros(max(n, 1), dtype=np.int32) for _ in range(3)]
    gain = np.zeros(max(n, 1), dtype=np.int64)
    M = lib().or_propose_moves(n, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.src_counts)),
                               _p(_i32(g.weights)), _p(_i32(size)), _p(_i32(rho)), nparts, omega,
                               int(second_half), _p(bufs[0]), _p(bufs[1]), _p(bufs[2]), _p(gain))
    return bufs[0][:M], bufs[1][:M], bufs[2][:M], gain[:M]


def sequence(g, size, nparts, node, src, dst, gain, window=256, rounds=16):
    M = len(node)
    seq = np.zeros(max(M, 1), dtype=np.int32)
    lib().or_sequence(g.num_nodes, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.src_counts)),
                      _p(_i32(size)), nparts, M, _p(_i32(node)), _p(_i32(src)), _p(_i32(dst)),
                      _p(np.ascontiguousarray(gain, dtype=np.int64)), window, rounds, _p(seq))
    return seq[:M]


def inseq_and_prefix(g, size, rho, nparts, node, dst, omega, delta):
    M = len(node)
    gseq = np.zeros(max(M, 1), dtype=np.int64)
    bg = ctypes.c_int64(0)
    k = lib().or_inseq_and_prefix(g.num_nodes, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)),
                                  _p(_i32(g.src_counts)), _p(_i32(g.weights)), _p(_i32(size)), _p(_i32(rho)),
                                  nparts, M, _p(_i32(node)), _p(_i32(dst)), omega, delta, _p(gseq),
                                  ctypes.byref(bg))
    return gseq[:M], int(k), int(bg.value)


def refine_rep(g, size, rho, nparts, second_half, omega, delta, window=256, rounds=16):
    rho = np.ascontiguousarray(rho, dtype=np.int32).copy()
    k = lib().or_refine_rep(g.num_nodes, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)),
                            _p(_i32(g.src_counts)), _p(_i32(g.weights)), _p(_i32(size)), _p(rho), nparts,
                            int(second_half), omega, delta, window, rounds)
    return int(k), rho


# ---- learned merge priority ----
def mlp_scores(feat, model):
    """Scores of the integer MLP on feature rows feat[count, 16] (uint8)."""
    f = np.ascontiguousarray(feat, dtype=np.uint8).reshape(-1, 16)
    out = np.zeros(max(len(f), 1), dtype=np.int64)
    st = lib().or_mlp_scores(_p(f), len(f), _p(model_vector(model)), _p(out))
    if st != OK:
        raise ValueError("invalid model")
    return out[: len(f)]


def learned_level(g, size, omega, delta, level, candK, csK, pi, model):
    """Learned priority on one level graph: (features [n*K, 16], rank of the
    node in its candidate's list or -1 [n*K], C(n) [n*pi], eta [n*pi])."""
    n = g.num_nodes
    candK = np.ascontiguousarray(candK, dtype=np.int32)
    csK = np.ascontiguousarray(csK, dtype=np.uint64)
    K = candK.size // max(n, 1)
    feat = np.zeros((max(n * K, 1), 16), dtype=np.uint8)
    rank = np.zeros(max(n * K, 1), dtype=np.int32)
    cand = np.zeros(max(n * pi, 1), dtype=np.int32)
    cs = np.zeros(max(n * pi, 1), dtype=np.uint64)
    st = lib().or_learned_level(n, g.num_hedges, _p(_i32(g.offsets)), _p(_i32(g.pins)), _p(_i32(g.src_counts)),
                                _p(_i32(size)), omega, delta, level, K, _p(candK), _p(csK), pi,
                                _p(model_vector(model)), _p(feat), _p(rank), _p(cand), _p(cs))
    if st != OK:
        raise ValueError(f"or_learned_level: status {st}")
    return feat[: n * K], rank[: n * K], cand[: n * pi], cs[: n * pi]


def log_code(x: int) -> int:
    return int(lib().or_log_code(ctypes.c_uint64(x)))
