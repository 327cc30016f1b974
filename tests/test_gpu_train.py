"""GPU training kernels of the learned merge priority against the fp64
reference (oracle/merge_train.py), the level-0 feature extraction against
the oracle, and a short training run that must learn a separable rule."""
import numpy as np
import pytest

import oracle
from oracle import merge_train as mt
from paper_2605_20497_gb300 import hp, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_20497_gb300 import build
    build.build()
    oracle.build()
    hp.load()
    return t


def close(a, b, rel):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.max(np.abs(a - b)) <= rel * max(np.max(np.abs(b)), 1e-30) + 1e-12


@pytest.mark.parametrize("count", [1, 31, 33, 4097, 100_000])
def test_gradient_matches_fp64_reference(torch, count):
    r = np.random.default_rng(count)
    feat = r.integers(0, 256, size=(count, 16)).astype(np.uint8)
    y = r.random(count).astype(np.float32)
    p = mt.random_params(count % 7).astype(np.float32)
    fd, yd, pd = (torch.from_numpy(a).cuda() for a in (feat, y, p))
    rc, g, loss = hp.merge_grad(fd, yd, pd)
    assert rc == hp.HP_OK, hp.hp_last_error()
    # the tensor-core form: bf16 operands of the five matrix products, fp32 sums
    lref, gref = mt.loss_and_grad(p.astype(np.float64), feat, y.astype(np.float64), mixed=True)
    assert loss == pytest.approx(lref, rel=1e-4)
    g = g.cpu().numpy()
    # per tensor, relative to its largest entry: fp32 sums over up to 10^5
    # rows, and the rare bf16 operand whose fp32 value falls on the other
    # side of a rounding boundary than its fp64 value (one bf16 step, 2^-8)
    for lo, hi in [(0, 1024), (1024, 1088), (1088, 5184), (5184, 5248), (5248, 5312), (5312, 5313)]:
        assert close(g[lo:hi], gref[lo:hi], 2e-3), (count, lo)
    rc2, g2, loss2 = hp.merge_grad(fd, yd, pd)
    assert np.array_equal(g, g2.cpu().numpy()) and loss == loss2   # fixed reduction order


def test_adam_matches_reference(torch):
    r = np.random.default_rng(5)
    p, g = r.normal(size=(2, hp.HP_MERGE_NPARAM)).astype(np.float32)
    m, v = (np.abs(r.normal(size=(2, hp.HP_MERGE_NPARAM))) * 0.01).astype(np.float32)
    t = [torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v)]
    assert hp.merge_adam(t[0], t[1], t[2], t[3], 7, lr=0.01, weight_decay=0.01) == hp.HP_OK
    torch.cuda.synchronize()
    # the kernel takes its hyperparameters in fp32: 1 - fp32(0.999) differs from 0.001 by 1.3e-5
    f = lambda x: float(np.float32(x))
    q, m2, v2 = mt.adamw_step(p, g, m, v, 7, f(0.01), f(0.9), f(0.999), f(1e-8), f(0.01))
    assert np.allclose(t[0].cpu().numpy(), q, rtol=1e-5, atol=1e-6)
    assert np.allclose(t[2].cpu().numpy(), m2, rtol=1e-5, atol=1e-7)
    assert np.allclose(t[3].cpu().numpy(), v2, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("case", range(3))
def test_level0_features_match_oracle(torch, case):
    extra = {}
    if case == 0:
        g, om, de = inputs.random_snn(2000, 15, seed=2), 16, 80
    elif case == 1:
        g, om, de = inputs.random_hypergraph(1500, 2200, 30, seed=3, multi_src=True, weights=True), 12, 70
    else:
        g, om, de, extra = inputs.random_snn(1200, 9, seed=4), 16, 120, dict(count_kind=1)
    K, seed = 16, 7
    rc, cand, rank, feat = hp.merge_features(g, om, de, seed=seed, learned_k=K, **extra)
    assert rc == hp.HP_OK, hp.hp_last_error()
    gg = g
    if extra.get("count_kind") == 1:   # every pin is a destination for the constraint
        gg = inputs.Hypergraph(num_nodes=g.num_nodes, offsets=g.offsets, pins=g.pins,
                               src_counts=np.zeros(g.num_hedges, np.int32), weights=g.weights)
    size = np.ones(g.num_nodes, np.int32)
    candK, csK = oracle.propose(gg, size, om, de, seed=seed, level=0, pi=K)
    of, orank, _, _ = oracle.learned_level(gg, size, om, de, 0, candK.ravel(), csK.ravel(), 4,
                                           inputs.constant_merge_model(0))
    assert np.array_equal(cand.cpu().numpy(), candK.ravel())
    assert np.array_equal(rank.cpu().numpy(), orank)
    assert np.array_equal(feat.cpu().numpy(), of)


def test_training_learns_a_separable_rule(torch):
    r = np.random.default_rng(11)
    feat = r.integers(0, 256, size=(50_000, 16)).astype(np.uint8)
    y = ((feat[:, 3].astype(int) + feat[:, 9]) > 255).astype(np.float32)
    fd, yd = torch.from_numpy(feat).cuda(), torch.from_numpy(y).cuda()
    p = torch.from_numpy(mt.random_params(0).astype(np.float32)).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    losses = []
    for step in range(1, 301):
        idx = torch.from_numpy(r.integers(0, len(y), 4096)).cuda()
        rc, g, loss = hp.merge_grad(fd[idx], yd[idx], p)
        assert rc == hp.HP_OK
        assert hp.merge_adam(p, g, m, v, step, lr=3e-3) == hp.HP_OK
        losses.append(loss)
    assert losses[0] > 0.5 and np.mean(losses[-20:]) < 0.25, (losses[0], losses[-20:])
    rc, model = hp.merge_quantize(p.cpu().numpy(), feat[:8192])
    assert rc == hp.HP_OK
    s = oracle.mlp_scores(feat, model)
    o = mt.forward(p.cpu().numpy().astype(np.float64), feat)[-1]
    assert np.mean((s > np.median(s)) == (o > np.median(o))) > 0.95


def test_trained_priority_gains_on_held_out_graphs(torch):
    """The committed model (trained by train_merge on 64 random SNN
    hypergraphs of 16,384 nodes, generator seeds 1..64) against the plain
    priority on held-out graphs of the same generator (seeds 100..102): the
    learned priority's connectivity is at most the plain one on each, with no
    Omega/Delta violation.  Partitions are bit-exact and deterministic, so
    this compares fixed numbers."""
    import os
    from paper_2605_20497_gb300 import train_merge
    path = os.path.join(os.path.dirname(hp.__file__), "merge_random_snn_16k.npz")
    model = train_merge.load(path)
    gains = []
    for s in (100, 101, 102):
        g = inputs.random_snn(16384, 127, seed=s)
        d = hp.to_device(g)
        a = hp.partition(g, 1024, 4096, seed=0, dev=d)
        b = hp.partition(g, 1024, 4096, seed=0, dev=d, learned_k=16, model=model)
        assert a.status == b.status == hp.HP_OK, hp.hp_last_error()
        assert b.stats["violations"] == 0
        assert b.stats["connectivity"] <= a.stats["connectivity"], (s, b.stats["connectivity"], a.stats["connectivity"])
        gains.append(a.stats["connectivity"] - b.stats["connectivity"])
    assert sum(gains) > 0
