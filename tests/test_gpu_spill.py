"""GPU decide/solve with the finished levels kept in pinned host memory
(spill_levels): the same level sets, fingerprints, counters and valid
orderings as the oracle, and a run that fits the device cap only this way."""
import json
import os

import pytest

import oracle
from oracle import bounds as obounds
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import assert_decide_matches, context

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_spilled_levels_match_oracle():
    # 32-, 64- and 128-bit states; orders are checked by assert_decide_matches
    cases = [gg.workload_gnp20(), gg.gnp(28, 0.25, 9), gg.partial_ktree(26, 5, 3), gg.relabel(gg.path(70), 5)]
    with context(fingerprints=True, spill_levels=True) as c:
        for adj in cases:
            lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
            tw = oracle.solve(adj, k_start=lb, want_order=False)["tw"]
            for k in sorted({max(0, tw - 1), tw}):
                assert_decide_matches(c, adj, k)


def test_spilled_solve_gives_a_valid_decomposition():
    adj = gg.partial_ktree(24, 6, 4)
    with context(spill_levels=True) as c:
        res = c.solve(adj, want_td=True)
    exp = oracle.solve(adj, k_start=max(obounds.mmd(adj), obounds.mmd_plus(adj)), want_order=False)["tw"]
    assert res["tw"] == exp
    assert oracle.width_elim(adj, res["order"].tolist()) == exp
    assert oracle.verify_td(adj, res["td_parent"], res["td_bags"]) == exp


def test_spill_fits_a_cap_the_resident_levels_exceed():
    # Every level of the k = 6 run of the n=40 geometric graph kept on the
    # device needs about 0.72 GB; alternating two levels and the table needs
    # well under 0.6 GB.
    from paper_1709_09990_gb300 import native
    adj = gg.workload_rgg40()
    rec = json.load(open(os.path.join(GOLDEN, "rgg40_seed0_k6.json")))["decide"][0]
    cap = 600 << 20
    with context(mem_cap_bytes=cap) as c:
        with pytest.raises(native.TwError) as e:
            c.decide(adj, k=6, want_order=True)
        assert e.value.status == native.TW_ERR_CAPACITY
    with context(mem_cap_bytes=cap, spill_levels=True, fingerprints=True) as c:
        got = c.decide(adj, k=6, want_order=True)
    assert got["yes"]
    assert got["stats"]["level_size"] == rec["level_size"]
    assert [str(x) for x in got["stats"]["fp_xor"]] == rec["fp_xor"]
    assert got["stats"]["peak_frontier_bytes"] < cap
    assert oracle.width_q(adj, got["order"].tolist()) <= 6


def test_batch_with_spilled_levels():
    # the geometric n=40 graph leaves the batch for the single-graph path,
    # which keeps its levels in host memory here
    graphs = [gg.workload_gnp20(), gg.workload_rgg40(), gg.cycle(12), gg.partial_ktree(24, 6, 4)]
    with context(spill_levels=True) as c:
        res = c.solve_batch(graphs)
    assert res["status"] == 0
    assert res["tw"].tolist() == [8, 6, 2, 6]
    pos = 0
    for adj, tw in zip(graphs, res["tw"].tolist()):
        assert oracle.width_q(adj, res["orders"][pos: pos + len(adj)].tolist()) == tw
        pos += len(adj)
