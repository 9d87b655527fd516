"""Writes tests/golden/grid53_plan.json: the contraction order and sliced
labels that the benchmark contracts the 53-qubit grid amplitude with, produced
by the library's host-side planner (greedy path, 512 trials, seed 1; slice
finder to 2^28 elements; slice-aware sub-tree reconfiguration, 8 passes).

The file is test INPUT, not an expected value: an order of pairwise steps
(Section 2.3: any order gives the same contraction) and a set of labels to fix
(Section 2.4: which partial sums s_i exist).  make_golden.py hands both to the
FP64 oracle as data; the oracle's own greedy order cannot contract this slicing
(its largest intermediate would be 2^41 elements).  No device is touched.

Usage: python tests/golden/make_plan.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from circuits import configs  # noqa: E402
from paper_2107_09793_b300 import jet  # noqa: E402

GRID53_PLAN = dict(seed=1, n_trials=512, cap=1 << 28, reconfigure_passes=8)


def plan_grid53():
    w = configs.build("grid53")
    net = jet.from_network(w.network, precision="fp32")
    t0 = time.time()
    net.path_greedy(seed=GRID53_PLAN["seed"], n_trials=GRID53_PLAN["n_trials"])
    sliced = net.slice_auto(GRID53_PLAN["cap"], min_n=0, max_n=60)
    f_before, f_after = net.path_reconfigure(GRID53_PLAN["reconfigure_passes"])
    st = net.stats()
    rec = {"workload": "grid53", "planner": GRID53_PLAN, "path": [list(map(int, p)) for p in net.path_get()],
           "sliced_labels": [int(x) for x in sliced], "max_intermediate": int(st["max_intermediate"]),
           "flop_per_slice": st["flop_sliced"] / st["n_slices"], "flop_whole_amplitude_reuse": f_after,
           "flop_before_reconfiguration": f_before, "planner_s": round(time.time() - t0, 1)}
    net.close()
    return rec


if __name__ == "__main__":
    rec = plan_grid53()
    with open(os.path.join(HERE, "grid53_plan.json"), "w") as f:
        json.dump(rec, f)
    print({k: v for k, v in rec.items() if k != "path"})
