"""Pins of the fp64 training reference of the learned merge priority: its
analytic gradient against central finite differences of its loss, the loss
at closed-form points, and the AdamW step's first update; plus the
library's host-side quantisation (no GPU needed), which must keep the float
model's ranking of pairs."""
import ctypes

import numpy as np
import pytest

from oracle import merge_train as mt


def data(n, seed):
    r = np.random.default_rng(seed)
    return r.integers(0, 256, size=(n, 16)).astype(np.uint8), r.integers(0, 2, size=n).astype(np.float64)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    feat, y = data(40, seed)
    p = mt.random_params(seed)
    _, g = mt.loss_and_grad(p, feat, y)
    rng = np.random.default_rng(seed + 10)
    # every bias and w3 entry, and a sample of W1 and W2 entries
    idx = np.concatenate([np.arange(1024, 1088), np.arange(5184, mt.NPARAM), rng.choice(1024, 60, replace=False),
                          1088 + rng.choice(4096, 120, replace=False)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mt.NPARAM)
        e[i] = h
        fd = (mt.loss(p + e, feat, y) - mt.loss(p - e, feat, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_loss_closed_forms():
    feat, y = data(10, 3)
    p = np.zeros(mt.NPARAM)
    assert mt.loss(p, feat, y) == pytest.approx(np.log(2.0))   # o = 0 everywhere
    p[-1] = 3.0                                                  # o = b3 = 3
    want = np.mean(np.where(y == 1, np.log1p(np.exp(-3.0)), 3.0 + np.log1p(np.exp(-3.0))))
    assert mt.loss(p, feat, y) == pytest.approx(want)
    l, g = mt.loss_and_grad(p, feat, y)
    assert g[-1] == pytest.approx(np.mean(1 / (1 + np.exp(-3.0)) - y))
    assert np.all(g[:-1] == 0)   # every hidden unit is dead


def test_adamw_first_step():
    # first step: m_hat = g, v_hat = g^2, so each parameter moves by lr * sign(g) (eps -> 0), plus decay
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    q, m, v = mt.adamw_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01, 0.9, 0.999, 1e-12, 0.1)
    assert np.allclose(q, p - 0.01 * (np.sign(g) + 0.1 * p))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


@pytest.fixture(scope="module")
def lib():
    from paper_2605_20497_gb300 import build, hp
    build.build()
    return hp.load()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quantised_model_keeps_the_ranking(lib, seed):
    import oracle
    from paper_2605_20497_gb300 import hp
    feat, _ = data(3000, seed)
    p = mt.random_params(seed).astype(np.float32)
    rc, model = hp.merge_quantize(p, feat[:2000])
    assert rc == hp.HP_OK
    s = oracle.mlp_scores(feat, model)                    # integer model
    o = mt.forward(p.astype(np.float64), feat)[-1]         # float model
    rank = lambda a: np.argsort(np.argsort(a, kind="stable"), kind="stable")
    rho = np.corrcoef(rank(s), rank(o))[0, 1]
    assert rho > 0.97, rho
    assert -127 <= model.w1.min() and model.w2.max() <= 127 and 0 <= model.shift1 <= 30


def test_quantise_checks_arguments(lib):
    from paper_2605_20497_gb300 import hp
    p = np.full(mt.NPARAM, np.nan, dtype=np.float32)
    rc, _ = hp.merge_quantize(p, np.zeros((4, 16), np.uint8))
    assert rc == hp.HP_ERR_INVALID_ARG
    rc, _ = hp.merge_quantize(np.zeros(mt.NPARAM, np.float32), np.zeros((0, 16), np.uint8))
    assert rc == hp.HP_ERR_INVALID_ARG


def test_model_file_round_trip_and_init(tmp_path):
    from paper_2605_20497_gb300 import inputs, train_merge
    m = inputs.random_merge_model(4)
    path = str(tmp_path / "m.npz")
    train_merge.save(path, m)
    back = train_merge.load(path)
    for k in ("w1", "w2", "w3", "b1", "b2"):
        assert np.array_equal(getattr(m, k), getattr(back, k)), k
    assert (back.b3, back.shift1, back.shift2) == (m.b3, m.shift1, m.shift2)
    p = train_merge.init_params(3)
    assert p.dtype == np.float32 and p.size == mt.NPARAM
    assert np.array_equal(p, train_merge.init_params(3)) and not np.array_equal(p, train_merge.init_params(4))
    assert p[-1] == 0.0 and np.all(np.abs(p[:1024]) <= np.sqrt(6 / 16))


def test_shipped_model_is_valid():
    import os
    import oracle
    from paper_2605_20497_gb300 import train_merge
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2605_20497_gb300",
                        "merge_random_snn_16k.npz")
    m = train_merge.load(path)
    s = oracle.mlp_scores(np.random.default_rng(0).integers(0, 256, size=(100, 16)).astype(np.uint8), m)
    assert len(np.unique(s)) > 10   # not a constant model


def test_bf16_rounding_pins():
    # round to nearest, ties to even, on the 8-bit significand of bfloat16
    x = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, 1 + 2**-7, -(2 + 2**-7 + 2**-9), 3.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2**-6, 1 + 2**-7, -(2 + 2**-6), 3.0, 0.0])
    assert np.array_equal(mt.bf16(x), want)


@pytest.mark.parametrize("seed", range(3))
def test_mixed_form_is_the_same_function_up_to_bf16(seed):
    r = np.random.default_rng(seed)
    feat = r.integers(0, 256, size=(300, 16))
    y = r.random(300)
    p = mt.random_params(seed)
    l0, g0 = mt.loss_and_grad(p, feat, y)
    l1, g1 = mt.loss_and_grad(p, feat, y, mixed=True)
    assert abs(l1 - l0) <= 1e-2 * abs(l0)
    assert np.max(np.abs(g1 - g0)) <= 3e-2 * np.max(np.abs(g0))
    # parameters and features that are exact bf16 with exact products leave
    # the forward pass unchanged
    q = mt.bf16(p)
    assert np.array_equal(mt.bf16(q), q)
    x1 = mt.forward(q, feat[:, :], mixed=False)
    assert np.allclose(x1[1], mt.forward(q, feat, mixed=True)[1])
