"""Writes the oracle's full-size results used by tests/test_gpu_fullsize.py.

Runs only the CPU oracle (oracle/) on full-size workloads whose generators
give the same input on every machine (the layered networks use no random
numbers; the random one draws from a SplitMix64 counter stream) and stores,
per workload: a hash of the generated input, the status, the statistics,
the per-level trace and a hash of the part vector.  A name ending in
"+learned" runs the learned merge priority (top-16 lists) with the seeded
random model inputs.random_merge_model(LEARNED_MODEL_SEED).  Usage (from the
repository root): python tests/golden/make_oracle_golden.py [workload ...]
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2605_20497_gb300 import inputs  # noqa: E402

STAT_KEYS = ("connectivity", "cut_net", "num_parts", "max_part_size", "max_part_distinct", "violations", "levels",
             "moves_applied")
TRACE_KEYS = ("n", "pins", "pairs", "iso_pairs", "conn", "moves", "reps", "valid", "iso_list", "targets_r1",
              "max_indeg_r1", "pairs_r1")
LEARNED_SUFFIX, LEARNED_K, LEARNED_MODEL_SEED = "+learned", 16, 7


def input_hash(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.offsets, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.pins, dtype="<i4").tobytes())
    return h.hexdigest()


def part_hash(part) -> str:
    return hashlib.sha256(np.ascontiguousarray(part, dtype="<i4").tobytes()).hexdigest()


def main(names):
    oracle.build()
    for name in names:
        learned = name.endswith(LEARNED_SUFFIX)
        base = name[: -len(LEARNED_SUFFIX)] if learned else name
        g = inputs.workload(base)
        om, de = inputs.CONSTRAINTS[base]
        opts = dict(learned_k=LEARNED_K, model=inputs.random_merge_model(LEARNED_MODEL_SEED)) if learned else {}
        t = time.time()
        r = oracle.partition(g, om, de, seed=0, trace=True, **opts)
        dt = time.time() - t
        out = {
            "workload": base, "omega": om, "delta": de, "seed": 0,
            "options": ({"learned_k": LEARNED_K, "random_merge_model_seed": LEARNED_MODEL_SEED} if learned
                        else "defaults"),
            "input_sha256": input_hash(g), "status": r.status,
            "stats": {k: int(r.stats[k]) for k in STAT_KEYS},
            "trace": [{k: int(lv[k]) for k in TRACE_KEYS} for lv in r.trace],
            "part_sha256": part_hash(r.part),
        }
        fname = f"oracle_{base}_learned.json" if learned else f"oracle_{name}.json"
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), fname)
        with open(path, "w") as f:
            json.dump(out, f, indent=0)
        print(name, "oracle %.1f s" % dt, out["stats"])


if __name__ == "__main__":
    main(sys.argv[1:] or ["layered_snn_65k", "layered_snn_262k", "random_snn_16k"])
