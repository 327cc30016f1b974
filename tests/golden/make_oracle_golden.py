"""Writes the oracle's full-size results used by tests/test_gpu_fullsize.py.

Runs only the CPU oracle (oracle/) on full-size workloads whose generators
give the same input on every machine (the layered networks use no random
numbers; the random one draws from a SplitMix64 counter stream) and stores,
per workload: a hash of the generated input, the status, the statistics,
the per-level trace and a hash of the part vector.  Usage (from the repository
root): python tests/golden/make_oracle_golden.py [workload ...]
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
TRACE_KEYS = ("n", "pins", "pairs", "iso_pairs", "conn", "moves", "reps")


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
        g = inputs.workload(name)
        om, de = inputs.CONSTRAINTS[name]
        t = time.time()
        r = oracle.partition(g, om, de, seed=0, trace=True)
        dt = time.time() - t
        out = {
            "workload": name, "omega": om, "delta": de, "seed": 0, "options": "defaults",
            "input_sha256": input_hash(g), "status": r.status,
            "stats": {k: int(r.stats[k]) for k in STAT_KEYS},
            "trace": [{k: int(lv[k]) for k in TRACE_KEYS} for lv in r.trace],
            "part_sha256": part_hash(r.part),
        }
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{name}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=0)
        print(name, "oracle %.1f s" % dt, out["stats"])


if __name__ == "__main__":
    main(sys.argv[1:] or ["layered_snn_65k", "layered_snn_262k", "random_snn_16k"])
