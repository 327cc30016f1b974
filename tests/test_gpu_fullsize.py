"""Full-size parity: the CUDA path on the layered spiking-network workloads
(65,536 and 262,144 nodes; the second is the one bench.py times, in the same
call configuration) and on the random one of 16,384 nodes with 127 targets
each (the 65k layered and the random one also with the learned merge
priority and a seeded random model),
against the oracle's results stored by
tests/golden/make_oracle_golden.py.  The oracle takes minutes on these, so
its part vector is compared by hash, with its statistics and its per-level
trace compared value by value."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2605_20497_gb300 import hp, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TRACE_KEYS = ("n", "pins", "pairs", "iso_pairs", "conn", "moves", "reps", "valid", "iso_list", "targets_r1",
              "max_indeg_r1", "pairs_r1")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_20497_gb300 import build
    build.build()
    hp.load()
    return t


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


@pytest.mark.parametrize("name", ["layered_snn_65k", "layered_snn_262k", "random_snn_16k", "random_snn_16k_learned",
                                  "layered_snn_65k_learned"])
def test_fullsize_matches_stored_oracle(torch, name):
    with open(os.path.join(GOLDEN, f"oracle_{name}.json")) as f:
        gold = json.load(f)
    g = inputs.workload(gold["workload"])
    opts = {}
    if isinstance(gold["options"], dict):
        opts = dict(learned_k=gold["options"]["learned_k"],
                    model=inputs.random_merge_model(gold["options"]["random_merge_model_seed"]))
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.offsets, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.pins, dtype="<i4").tobytes())
    assert h.hexdigest() == gold["input_sha256"], "the generator no longer builds the stored input"
    r = hp.partition(g, gold["omega"], gold["delta"], seed=gold["seed"], trace=True, **opts)
    assert r.status == gold["status"] == hp.HP_OK, hp.hp_last_error()
    for k, v in gold["stats"].items():
        assert r.stats[k] == v, (k, r.stats[k], v)
    assert len(r.trace) == len(gold["trace"])
    for lv, (a, b) in enumerate(zip(r.trace, gold["trace"])):
        for k in TRACE_KEYS:
            assert a[k] == b[k], (lv, k, a[k], b[k])
    assert sha(r.part) == gold["part_sha256"]
    # properties that hold at any size: every part within Omega and Delta
    assert r.stats["violations"] == 0
    assert r.stats["max_part_size"] <= gold["omega"]
