"""Writes the stored expected values under tests/golden/ from the CPU oracle.

Run from the repository root:  python tests/golden/make_golden.py
Every value written here comes from ``oracle/`` alone (the paper prints no
worked example for these synthetic inputs).  The test suite re-derives the
small ones with the independent subset DP.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1709_09990_gb300 import graphgen as gg  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def decide_record(adj, k):
    d = oracle.decide(adj, k, count_canonical=True)
    return {"k": k, "yes": d["yes"], "levels": d["levels"], "level_size": d["level_size"],
            "fp_sum": [str(x) for x in d["fp_sum"]], "fp_xor": [str(x) for x in d["fp_xor"]],
            "states_expanded": d["states_expanded"], "candidates": d["candidates"],
            "feasible": d["feasible"], "canonical": d["canonical"]}


def main():
    adj = gg.workload_gnp20()
    sol = oracle.solve(adj, 0, want_order=False)
    rec = {"workload": "G(n=20, p=0.3), seed 0", "n": 20, "tw": sol["tw"],
           "sweep_from_0": {"states_expanded": sol["states_expanded"], "candidates": sol["candidates"],
                            "feasible": sol["feasible"], "k_tried": sol["k_tried"]},
           "decide": [decide_record(adj, k) for k in range(0, sol["tw"] + 2)]}
    with open(os.path.join(HERE, "gnp20_seed0.json"), "w") as f:
        json.dump(rec, f, indent=1)
    # Level records of the random geometric graph at k = 4 and k = tw-1 = 5
    # (the largest "no" run); the k = tw = 6 run takes minutes in the oracle
    # and is written only with --full (below).
    adj = gg.workload_rgg40()
    rec = {"workload": "random geometric graph n=40, r=0.25, seed 0", "n": 40,
           "decide": [decide_record(adj, k) for k in (4, 5)]}
    with open(os.path.join(HERE, "rgg40_seed0_k4_k5.json"), "w") as f:
        json.dump(rec, f, indent=1)
    if "--full" in sys.argv:
        # The k = tw = 6 run of the same graph: about 78 million states, on the
        # order of ten minutes of oracle time on one core.
        rec = {"workload": "random geometric graph n=40, r=0.25, seed 0", "n": 40,
               "decide": [decide_record(adj, 6)]}
        with open(os.path.join(HERE, "rgg40_seed0_k6.json"), "w") as f:
            json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
