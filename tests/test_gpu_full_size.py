"""Parity on the benchmark workloads themselves, at their full sizes, where
the oracle cannot finish them: the first levels against the oracle run only
that far, and properties that hold at any size for the rest.  (The n=40
geometric graph is compared level by level in full in test_gpu_decide.)"""
import pytest

import oracle
from oracle import bounds as obounds
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


def test_partial_10tree_first_levels_match_oracle():
    # decide(10) on the partial 10-tree n=60 under a 4 GB cap stops with the
    # capacity status after level 8 (56.7 M states); levels 0..5 are the
    # oracle's, and the counters of every completed level are consistent.
    from paper_1709_09990_gb300 import native
    adj = gg.workload_pktree60()
    n, k = len(adj), 10
    with context(fingerprints=True, mem_cap_bytes=4 << 30) as c:
        with pytest.raises(native.TwError) as e:
            c.decide(adj, k=k)
    assert e.value.status == native.TW_ERR_CAPACITY
    st = e.value.stats
    exp = oracle.decide_prefix(adj, k, 5)
    assert st["level_size"][:6] == exp["level_size"]
    assert st["fp_sum"][:6] == exp["fp_sum"] and st["fp_xor"][:6] == exp["fp_xor"]
    sizes = st["level_size"]
    last = len(sizes) - 1
    assert last >= 8
    assert st["states_expanded"] == sum(sizes[:last])
    assert st["candidates"] == sum(s * (n - i) for i, s in enumerate(sizes[:last]))
    assert st["generated"] >= sum(sizes[1:])


def test_batch_workload_sample():
    # the first 256 graphs of the 4096-graph batch, as the benchmark solves
    # them (one batched call, 16 GB cap): every answered graph's ordering has
    # width exactly tw, and the small ones match the oracle's treewidth
    graphs = gg.batch_graphs(256)
    with context(mem_cap_bytes=16 << 30) as c:
        res = c.solve_batch(graphs)
    per = res["per_graph_status"].tolist()
    tw = res["tw"].tolist()
    assert sum(s == 0 for s in per) > 200
    pos = 0
    checked = 0
    for g, adj in enumerate(graphs):
        n = len(adj)
        if per[g] == 0:
            order = res["orders"][pos: pos + n].tolist()
            assert sorted(order) == list(range(n))
            assert oracle.width_q(adj, order) == tw[g]
            assert max(obounds.mmd(adj), obounds.mmd_plus(adj)) <= tw[g]
            if n <= 22:
                lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
                assert tw[g] == oracle.solve(adj, k_start=lb, want_order=False)["tw"], g
                checked += 1
        pos += n
    assert checked >= 30
