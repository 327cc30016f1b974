"""Thin ctypes binding of libhp.so (include/hp.h): argument marshalling only.

Every function named ``hp_*`` forwards to the C function of the same name.
Device buffers are plain integers (device addresses), e.g. from
``torch.Tensor.data_ptr()``; ``stream`` is a ``cudaStream_t`` as an integer
(``torch.cuda.current_stream().cuda_stream``) or 0.  :func:`partition` is a
convenience wrapper that moves a numpy CSR hypergraph to the GPU with torch,
calls :func:`hp_partition_ex` and returns numpy results.

There is no CPU fallback: :func:`load` raises when the library has not been
built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhp.so")

HP_OK, HP_ERR_INVALID_ARG, HP_ERR_BAD_CSR, HP_ERR_INFEASIBLE = 0, 1, 2, 3
HP_ERR_OOM, HP_ERR_CUDA, HP_ERR_TIMEOUT, HP_ERR_INTERNAL = 4, 5, 6, 7
HP_COUNT_INBOUND, HP_COUNT_INCIDENT = 0, 1

EXPORTS = ("hp_default_options", "hp_partition", "hp_partition_ex", "hp_partition_host", "hp_set_allocator",
           "hp_status_string", "hp_last_error", "hp_connectivity", "hp_connectivity_noalloc", "hp_partition_batch", "hp_merge_scores",
           "hp_merge_features", "hp_merge_grad", "hp_merge_adam", "hp_merge_quantize", "hp_debug_coarsen_level",
           "hp_debug_refine_rep", "hp_batch_tuned_concurrency")
HP_MERGE_NPARAM = 5313


class hp_merge_model(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_int8 * 1024), ("w2", ctypes.c_int8 * 4096), ("w3", ctypes.c_int8 * 64),
                ("b1", ctypes.c_int32 * 64), ("b2", ctypes.c_int32 * 64), ("b3", ctypes.c_int32),
                ("shift1", ctypes.c_int32), ("shift2", ctypes.c_int32)]


class hp_options(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("pi", "theta", "chain_window", "chain_rounds", "noise_permille",
                                               "count_kind", "max_levels", "debug_table_cap", "learned_k",
                                               "debug_walk_cap")] + [("merge_model", ctypes.POINTER(hp_merge_model)),
                                                                     ("node_batch", ctypes.c_int32),
                                                                     ("learned_levels", ctypes.c_int32)]


def merge_model(m) -> hp_merge_model:
    """ctypes hp_merge_model of an inputs.MergeModel."""
    x = hp_merge_model()
    ctypes.memmove(x.w1, np.ascontiguousarray(m.w1, dtype=np.int8).ctypes.data, 1024)
    ctypes.memmove(x.w2, np.ascontiguousarray(m.w2, dtype=np.int8).ctypes.data, 4096)
    ctypes.memmove(x.w3, np.ascontiguousarray(m.w3, dtype=np.int8).ctypes.data, 64)
    ctypes.memmove(x.b1, np.ascontiguousarray(m.b1, dtype=np.int32).ctypes.data, 256)
    ctypes.memmove(x.b2, np.ascontiguousarray(m.b2, dtype=np.int32).ctypes.data, 256)
    x.b3, x.shift1, x.shift2 = int(m.b3), int(m.shift1), int(m.shift2)
    return x


class hp_stats(ctypes.Structure):
    _fields_ = [("connectivity", ctypes.c_int64), ("cut_net", ctypes.c_int64), ("num_parts", ctypes.c_int32),
                ("max_part_size", ctypes.c_int32), ("max_part_distinct", ctypes.c_int32),
                ("violations", ctypes.c_int32), ("levels", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("moves_applied", ctypes.c_int64), ("pin_visits", ctypes.c_int64), ("ms_total", ctypes.c_double),
                ("ms_coarsen", ctypes.c_double), ("ms_refine", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("l0_pin_visits", ctypes.c_int64),
                ("l0_neighbours", ctypes.c_int64), ("ms_propose_l0", ctypes.c_double), ("alg_bytes", ctypes.c_int64)]


class hp_level_trace(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pairs", ctypes.c_int32), ("iso_pairs", ctypes.c_int32),
                ("reps", ctypes.c_int32), ("pins", ctypes.c_int64), ("conn", ctypes.c_int64),
                ("moves", ctypes.c_int64), ("valid", ctypes.c_int32), ("iso_list", ctypes.c_int32),
                ("targets_r1", ctypes.c_int32), ("max_indeg_r1", ctypes.c_int32), ("pairs_r1", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class hp_instance(ctypes.Structure):
    _fields_ = [("pins", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("src_counts", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("num_hedges", ctypes.c_int32), ("num_nodes", ctypes.c_int32),
                ("omega", ctypes.c_int32), ("delta", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("part_out", ctypes.c_void_p)]


_lib = None
P, I32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64


def load() -> ctypes.CDLL:
    """Load libhp.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2605_20497_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.hp_default_options.argtypes = [ctypes.POINTER(hp_options)]
        L.hp_default_options.restype = None
        part_args = [P, P, I32, I32, P, P, I32, I32, U64, ctypes.POINTER(hp_options), P, ctypes.POINTER(hp_stats)]
        L.hp_partition.argtypes = part_args + [P]
        L.hp_partition.restype = ctypes.c_int
        L.hp_partition_ex.argtypes = part_args + [ctypes.POINTER(hp_level_trace), I32, P]
        L.hp_partition_ex.restype = ctypes.c_int
        L.hp_partition_host.argtypes = part_args + [P]
        L.hp_partition_host.restype = ctypes.c_int
        L.hp_set_allocator.argtypes = [P, P, P]
        L.hp_set_allocator.restype = ctypes.c_int
        L.hp_status_string.argtypes = [ctypes.c_int]
        L.hp_status_string.restype = ctypes.c_char_p
        L.hp_last_error.argtypes = []
        L.hp_last_error.restype = ctypes.c_char_p
        L.hp_connectivity.argtypes = [P, P, I32, P, P, I32, I32, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), P]
        L.hp_connectivity.restype = ctypes.c_int
        L.hp_partition_batch.argtypes = [ctypes.POINTER(hp_instance), I32, ctypes.POINTER(hp_options), I32,
                                         ctypes.POINTER(hp_stats), ctypes.POINTER(ctypes.c_int32), P]
        L.hp_partition_batch.restype = ctypes.c_int
        L.hp_batch_tuned_concurrency.argtypes = [I32, I32]
        L.hp_batch_tuned_concurrency.restype = I32
        L.hp_merge_scores.argtypes = [P, ctypes.c_int64, ctypes.POINTER(hp_merge_model), P, P]
        L.hp_merge_scores.restype = ctypes.c_int
        L.hp_merge_features.argtypes = [P, P, I32, I32, P, P, I32, I32, U64, ctypes.POINTER(hp_options), P, P, P, P]
        L.hp_merge_features.restype = ctypes.c_int
        L.hp_merge_grad.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.POINTER(ctypes.c_double), P]
        L.hp_merge_grad.restype = ctypes.c_int
        F = ctypes.c_float
        L.hp_merge_adam.argtypes = [P, P, P, P, ctypes.c_int64, F, F, F, F, F, P]
        L.hp_merge_adam.restype = ctypes.c_int
        L.hp_merge_quantize.argtypes = [P, P, ctypes.c_int64, ctypes.POINTER(hp_merge_model)]
        L.hp_merge_quantize.restype = ctypes.c_int
        L.hp_connectivity_noalloc.argtypes = L.hp_connectivity.argtypes
        L.hp_connectivity_noalloc.restype = ctypes.c_int
        L.hp_debug_coarsen_level.argtypes = [I32, I32, P, P, P, P, P, I32, I32, U64, I32, ctypes.POINTER(hp_options),
                                             P, P, P, ctypes.POINTER(ctypes.c_int64), P]
        L.hp_debug_coarsen_level.restype = ctypes.c_int
        L.hp_debug_refine_rep.argtypes = [I32, I32, P, P, P, P, P, P, I32, I32, I32, I32,
                                          ctypes.POINTER(hp_options), P, P, P, P, P, P,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64), P]
        L.hp_debug_refine_rep.restype = ctypes.c_int
        _lib = L
    return _lib


# ------------------------------------------------------------- same-name calls
def hp_default_options() -> hp_options:
    o = hp_options()
    load().hp_default_options(ctypes.byref(o))
    return o


def hp_partition(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta, seed, opt, part_out,
                 stats, stream=0) -> int:
    return load().hp_partition(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta,
                               ctypes.c_uint64(seed), opt, part_out, stats, stream)


def hp_partition_ex(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta, seed, opt, part_out,
                    stats, trace, trace_cap, stream=0) -> int:
    return load().hp_partition_ex(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta,
                                  ctypes.c_uint64(seed), opt, part_out, stats, trace, trace_cap, stream)


def hp_partition_host(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta, seed, opt, part_out,
                      stats, stream=0) -> int:
    return load().hp_partition_host(pins, offsets, num_hedges, num_nodes, src_counts, weights, omega, delta,
                                    ctypes.c_uint64(seed), opt, part_out, stats, stream)


def hp_connectivity(pins, offsets, num_hedges, weights, part, num_nodes, num_parts, stream=0):
    c, cn = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().hp_connectivity(pins, offsets, num_hedges, weights, part, num_nodes, num_parts, ctypes.byref(c),
                                ctypes.byref(cn), stream)
    return st, int(c.value), int(cn.value)


def hp_connectivity_noalloc(pins, offsets, num_hedges, weights, part, num_nodes, num_parts, stream=0):
    c, cn = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().hp_connectivity_noalloc(pins, offsets, num_hedges, weights, part, num_nodes, num_parts,
                                        ctypes.byref(c), ctypes.byref(cn), stream)
    return st, int(c.value), int(cn.value)


def hp_debug_coarsen_level(num_nodes, num_hedges, offsets, pins, src_counts, weights, size, omega, delta, seed,
                           level, opt, cand_out, score_out, mate_out, stream=0):
    pairs = ctypes.c_int64(0)
    st = load().hp_debug_coarsen_level(num_nodes, num_hedges, offsets, pins, src_counts, weights, size, omega,
                                       delta, ctypes.c_uint64(seed), level, opt, cand_out, score_out, mate_out,
                                       ctypes.byref(pairs), stream)
    return st, int(pairs.value)


def hp_debug_refine_rep(num_nodes, num_hedges, offsets, pins, src_counts, weights, size, rho, num_parts,
                        second_half, omega, delta, opt, move_node, move_src, move_dst, move_gain, seq, gseq,
                        stream=0):
    m, k, bg = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    st = load().hp_debug_refine_rep(num_nodes, num_hedges, offsets, pins, src_counts, weights, size, rho,
                                    num_parts, second_half, omega, delta, opt, move_node, move_src, move_dst,
                                    move_gain, seq, gseq, ctypes.byref(m), ctypes.byref(k), ctypes.byref(bg),
                                    stream)
    return st, int(m.value), int(k.value), int(bg.value)


def hp_status_string(status: int) -> str:
    return load().hp_status_string(status).decode()


def hp_last_error() -> str:
    return load().hp_last_error().decode()


# ------------------------------------------------------------- convenience
@dataclass
class Result:
    status: int
    part: np.ndarray
    stats: dict
    trace: list


def options(model=None, **kw) -> hp_options:
    """hp_options from keyword values; ``model`` (an inputs.MergeModel) is
    converted and kept alive with the returned struct."""
    o = hp_default_options()
    for k, v in kw.items():
        setattr(o, k, int(v))
    if model is not None:
        o._model = merge_model(model)
        o.merge_model = ctypes.pointer(o._model)
    return o


def hp_merge_scores(feat, count, model, score_out, stream=0):
    return load().hp_merge_scores(feat, count, model, score_out, stream)


def merge_scores(feat, model, stream=0):
    """Scores of the learned priority's MLP for feature rows feat[count, 16]
    (uint8 torch tensor on the GPU); returns (status, int32 tensor)."""
    import torch
    count = feat.shape[0]
    out = torch.empty(max(count, 1), dtype=torch.int32, device=feat.device)
    m = merge_model(model)
    rc = hp_merge_scores(feat.data_ptr() if count else None, count, ctypes.byref(m),
                         out.data_ptr() if count else None, stream)
    torch.cuda.synchronize()
    return rc, out[:count]


def _stats_dict(s: hp_stats) -> dict:
    return {k: getattr(s, k) for k, _ in hp_stats._fields_ if k != "reserved0"}


def to_device(g, device="cuda"):
    """numpy CSR hypergraph -> dict of int32 torch tensors on the GPU."""
    import torch
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(device)
    return dict(offsets=t(g.offsets), pins=t(g.pins) if g.num_pins else torch.zeros(1, dtype=torch.int32, device=device),
                src_counts=t(g.src_counts), weights=t(g.weights))


def partition(g, omega: int, delta: int, seed: int = 0, trace: bool = False, dev=None, stream=0, **opts) -> Result:
    """Partition numpy hypergraph ``g`` on the current CUDA device."""
    import torch
    d = dev if dev is not None else to_device(g)
    part = torch.empty(max(g.num_nodes, 1), dtype=torch.int32, device=d["offsets"].device)
    st = hp_stats()
    cap = 4096 if trace else 0
    tr = (hp_level_trace * cap)() if cap else None
    ptr = lambda x: None if x is None else x.data_ptr()
    rc = hp_partition_ex(ptr(d["pins"]), ptr(d["offsets"]), g.num_hedges, g.num_nodes, ptr(d["src_counts"]),
                         ptr(d["weights"]), omega, delta, seed, ctypes.byref(options(**opts)), part.data_ptr(),
                         ctypes.byref(st), tr, cap, stream)
    torch.cuda.synchronize()
    sd = _stats_dict(st)
    levels = []
    if rc == HP_OK and tr is not None:
        for l in range(min(sd["levels"], cap)):
            x = tr[l]
            levels.append(dict(n=x.n, pins=x.pins, pairs=x.pairs, iso_pairs=x.iso_pairs, conn=x.conn,
                               moves=x.moves, reps=x.reps, valid=x.valid, iso_list=x.iso_list,
                               targets_r1=x.targets_r1, max_indeg_r1=x.max_indeg_r1, pairs_r1=x.pairs_r1))
    return Result(rc, part[: g.num_nodes].cpu().numpy(), sd, levels)


def partition_host(g, omega: int, delta: int, seed: int = 0, stream=0, **opts) -> Result:
    """Host-memory entry point: one copy in, one copy out (hp_partition_host)."""
    a = lambda x: None if x is None else np.ascontiguousarray(x, dtype=np.int32)
    off, pins, src, w = a(g.offsets), a(g.pins), a(g.src_counts), a(g.weights)
    part = np.zeros(max(g.num_nodes, 1), dtype=np.int32)
    st = hp_stats()
    p = lambda x: None if x is None else x.ctypes.data
    rc = hp_partition_host(p(pins), p(off), g.num_hedges, g.num_nodes, p(src), p(w), omega, delta, seed,
                           ctypes.byref(options(**opts)), p(part), ctypes.byref(st), stream)
    return Result(rc, part[: g.num_nodes], _stats_dict(st), [])


def partition_batch(graphs, concurrency: int = 8, stream=0, **opts):
    """graphs: list of (Hypergraph, omega, delta, seed).  Returns (status,
    [Result]) from one hp_partition_batch call on device copies."""
    import torch
    n = len(graphs)
    devs, parts = [], []
    arr = (hp_instance * max(n, 1))()
    for i, (g, om, de, seed) in enumerate(graphs):
        d = to_device(g)
        part = torch.empty(max(g.num_nodes, 1), dtype=torch.int32, device="cuda")
        devs.append(d)
        parts.append(part)
        ptr = lambda x: None if x is None else x.data_ptr()
        arr[i] = hp_instance(ptr(d["pins"]), ptr(d["offsets"]), ptr(d["src_counts"]), ptr(d["weights"]), g.num_hedges,
                             g.num_nodes, om, de, seed & (2**64 - 1), part.data_ptr())
    st = (hp_stats * max(n, 1))()
    ss = (ctypes.c_int32 * max(n, 1))()
    rc = load().hp_partition_batch(arr, n, ctypes.byref(options(**opts)), concurrency, st, ss, stream)
    torch.cuda.synchronize()
    out = [Result(int(ss[i]), parts[i][: graphs[i][0].num_nodes].cpu().numpy(), _stats_dict(st[i]), [])
           for i in range(n)]
    return rc, out


# ------------------------------------------------------------- learned priority training
def merge_features(g, omega: int, delta: int, seed: int = 0, learned_k: int = 16, dev=None, stream=0, **opts):
    """Level-0 training rows of hypergraph g (hp_merge_features): returns
    (status, cand, rank, feat) as GPU tensors of num_nodes*K entries."""
    import torch
    d = dev if dev is not None else to_device(g)
    n, K = g.num_nodes, learned_k
    cand = torch.empty(max(n * K, 1), dtype=torch.int32, device="cuda")
    rank = torch.empty(max(n * K, 1), dtype=torch.int32, device="cuda")
    feat = torch.empty((max(n * K, 1), 16), dtype=torch.uint8, device="cuda")
    ptr = lambda x: None if x is None else x.data_ptr()
    o = options(learned_k=K, **opts)
    rc = load().hp_merge_features(ptr(d["pins"]), ptr(d["offsets"]), g.num_hedges, n, ptr(d["src_counts"]),
                                  ptr(d["weights"]), omega, delta, seed & (2**64 - 1), ctypes.byref(o),
                                  cand.data_ptr(), rank.data_ptr(), feat.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, cand[: n * K], rank[: n * K], feat[: n * K]


def merge_grad(feat, label, params, stream=0):
    """(status, grad, mean loss) of the trainable form over rows feat[count,16]
    (uint8) with labels label[count] (float32); GPU tensors."""
    import torch
    count = feat.shape[0]
    grad = torch.empty(HP_MERGE_NPARAM, dtype=torch.float32, device=params.device)
    loss = ctypes.c_double(0.0)
    rc = load().hp_merge_grad(feat.data_ptr() if count else None, label.data_ptr() if count else None, count,
                              params.data_ptr(), grad.data_ptr(), ctypes.byref(loss), stream)
    return rc, grad, loss.value


def merge_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=0):
    return load().hp_merge_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), step, lr, beta1,
                                beta2, eps, weight_decay, stream)


def merge_quantize(params, calib):
    """(status, inputs.MergeModel) from float parameters (numpy float32
    [HP_MERGE_NPARAM]) and calibration rows (numpy uint8 [count, 16])."""
    from . import inputs
    p = np.ascontiguousarray(params, dtype=np.float32)
    c = np.ascontiguousarray(calib, dtype=np.uint8).reshape(-1, 16)
    m = hp_merge_model()
    rc = load().hp_merge_quantize(p.ctypes.data, c.ctypes.data if len(c) else None, len(c), ctypes.byref(m))
    out = inputs.MergeModel(
        w1=np.ctypeslib.as_array(m.w1).astype(np.int8).reshape(64, 16).copy(),
        w2=np.ctypeslib.as_array(m.w2).astype(np.int8).reshape(64, 64).copy(),
        w3=np.ctypeslib.as_array(m.w3).astype(np.int8).copy(),
        b1=np.ctypeslib.as_array(m.b1).astype(np.int32).copy(), b2=np.ctypeslib.as_array(m.b2).astype(np.int32).copy(),
        b3=int(m.b3), shift1=int(m.shift1), shift2=int(m.shift2))
    return rc, out
