"""Trains the learned merge priority and compares it with the paper's.

Every step runs in the library's CUDA kernels; this module only orders the
calls and moves the tensors:

1. plain partitions (``hp_partition``) of training hypergraphs give the
   labels: a level-0 candidate pair is positive when both ends end up in the
   same part;
2. ``hp_merge_features`` gives the features of every mutual level-0 pair, as
   the partitioner computes them;
3. minibatch AdamW (``hp_merge_grad``, ``hp_merge_adam``) fits the fp32 form
   of the MLP to the labels (binary cross-entropy);
4. ``hp_merge_quantize`` turns it into the integer model the partitioner
   runs;
5. held-out hypergraphs are partitioned with both priorities at the same
   Omega and Delta, and their connectivities (Eq. 1) are reported.

Usage: ``python -m paper_2605_20497_gb300.train_merge --out model.npz``
(defaults: 16,384-node random SNN hypergraphs with 127 targets per node,
Omega = 1024, Delta = 4096, training seeds 1..8, held-out seeds 100..102).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import hp, inputs


def init_params(seed: int) -> np.ndarray:
    """He-style uniform initialisation of the flat fp32 parameters."""
    r = np.random.default_rng(seed)
    w1 = r.uniform(-1, 1, (64, 16)) * np.sqrt(6 / 16)
    w2 = r.uniform(-1, 1, (64, 64)) * np.sqrt(6 / 64)
    w3 = r.uniform(-1, 1, 64) * np.sqrt(6 / 64)
    p = np.concatenate([w1.ravel(), r.uniform(-0.1, 0.1, 64), w2.ravel(), r.uniform(-0.1, 0.1, 64), w3, [0.0]])
    assert p.size == hp.HP_MERGE_NPARAM
    return p.astype(np.float32)


def dataset(graphs, K: int = 16):
    """(features [rows, 16] uint8, labels [rows] float32) on the GPU from the
    mutual level-0 pairs of every (hypergraph, Omega, Delta, seed)."""
    import torch
    feats, labels = [], []
    for g, om, de, sd in graphs:
        d = hp.to_device(g)
        r = hp.partition(g, om, de, seed=sd, dev=d)
        if r.status != hp.HP_OK:
            raise RuntimeError(hp.hp_last_error())
        part = torch.from_numpy(r.part).cuda()
        rc, cand, rank, feat = hp.merge_features(g, om, de, seed=sd, learned_k=K, dev=d)
        if rc != hp.HP_OK:
            raise RuntimeError(hp.hp_last_error())
        keep = rank >= 0
        v = torch.arange(g.num_nodes * K, device="cuda") // K
        same = part[v] == part[cand.clamp(min=0).long()]
        feats.append(feat[keep])
        labels.append(same[keep].float())
    return torch.cat(feats), torch.cat(labels)


def train(feat, label, steps: int = 400, batch: int = 65536, lr: float = 3e-3, weight_decay: float = 0.0,
          seed: int = 0):
    """Minibatch AdamW on the GPU; returns (params tensor, losses)."""
    import torch
    p = torch.from_numpy(init_params(seed)).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    r = np.random.default_rng(seed)
    losses = []
    n = feat.shape[0]
    for step in range(1, steps + 1):
        idx = torch.from_numpy(r.integers(0, n, size=min(batch, n))).cuda()
        rc, g, loss = hp.merge_grad(feat[idx], label[idx], p)
        if rc != hp.HP_OK:
            raise RuntimeError(hp.hp_last_error())
        if hp.merge_adam(p, g, m, v, step, lr=lr, weight_decay=weight_decay) != hp.HP_OK:
            raise RuntimeError(hp.hp_last_error())
        losses.append(loss)
    return p, losses


def compare(graphs, model, K: int = 16):
    """Connectivity and time of both priorities on each held-out graph."""
    rows = []
    for g, om, de, sd in graphs:
        d = hp.to_device(g)
        t0 = time.perf_counter()
        a = hp.partition(g, om, de, seed=sd, dev=d)
        t1 = time.perf_counter()
        b = hp.partition(g, om, de, seed=sd, dev=d, learned_k=K, model=model)
        t2 = time.perf_counter()
        if a.status != hp.HP_OK or b.status != hp.HP_OK:
            raise RuntimeError(hp.hp_last_error())
        rows.append({"graph": g.name, "omega": om, "delta": de, "plain_connectivity": a.stats["connectivity"],
                     "learned_connectivity": b.stats["connectivity"], "plain_parts": a.stats["num_parts"],
                     "learned_parts": b.stats["num_parts"], "learned_violations": b.stats["violations"],
                     "plain_ms": (t1 - t0) * 1e3, "learned_ms": (t2 - t1) * 1e3})
    return rows


def save(path: str, model: inputs.MergeModel):
    np.savez(path, w1=model.w1, w2=model.w2, w3=model.w3, b1=model.b1, b2=model.b2,
             b3=np.int32(model.b3), shift1=np.int32(model.shift1), shift2=np.int32(model.shift2))


def load(path: str) -> inputs.MergeModel:
    z = np.load(path)
    return inputs.MergeModel(w1=z["w1"], w2=z["w2"], w3=z["w3"], b1=z["b1"], b2=z["b2"], b3=int(z["b3"]),
                             shift1=int(z["shift1"]), shift2=int(z["shift2"]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, default=16384)
    ap.add_argument("--targets", type=int, default=127)
    ap.add_argument("--omega", type=int, default=1024)
    ap.add_argument("--delta", type=int, default=4096)
    ap.add_argument("--train-seeds", type=int, default=8, help="training hypergraphs (generator seeds 1..N)")
    ap.add_argument("--eval-seeds", type=int, default=3, help="held-out hypergraphs (generator seeds 100..)")
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    torch.cuda.init()
    mk = lambda s: (inputs.random_snn(args.nodes, args.targets, seed=s), args.omega, args.delta, 0)
    t0 = time.perf_counter()
    feat, label = dataset([mk(s) for s in range(1, args.train_seeds + 1)], args.k)
    t1 = time.perf_counter()
    p, losses = train(feat, label, args.steps, args.batch, args.lr)
    t2 = time.perf_counter()
    model_rc, model = hp.merge_quantize(p.cpu().numpy(), feat[: 1 << 16].cpu().numpy())
    if model_rc != hp.HP_OK:
        raise RuntimeError(hp.hp_last_error())
    rows = compare([mk(s) for s in range(100, 100 + args.eval_seeds)], model, args.k)
    out = {"rows": int(feat.shape[0]), "positive_fraction": float(label.mean().item()),
           "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:])), "dataset_s": t1 - t0,
           "train_s": t2 - t1, "steps": args.steps, "batch": args.batch, "eval": rows}
    if args.out:
        save(args.out, model)
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
