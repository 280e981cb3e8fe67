"""The stored oracle records under tests/golden/ still match the oracle, and
the small ones also match the independent subset DP."""
import json
import os

import oracle
from paper_1709_09990_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _same(rec, d):
    assert d["yes"] == rec["yes"]
    assert d["levels"] == rec["levels"]
    assert d["level_size"] == rec["level_size"]
    assert [str(x) for x in d["fp_sum"]] == rec["fp_sum"]
    assert [str(x) for x in d["fp_xor"]] == rec["fp_xor"]


def test_gnp20_golden():
    rec = _load("gnp20_seed0.json")
    adj = gg.workload_gnp20()
    assert oracle.solve(adj, want_order=False)["tw"] == rec["tw"]
    for r in rec["decide"]:
        _same(r, oracle.decide(adj, r["k"]))
        if r["k"] >= rec["tw"] - 1:
            _same(r, oracle.subset_dp(adj, r["k"]))


def test_rgg40_golden_small_k():
    rec = _load("rgg40_seed0_k4_k5.json")
    adj = gg.workload_rgg40()
    for r in rec["decide"]:
        _same(r, oracle.decide(adj, r["k"]))
