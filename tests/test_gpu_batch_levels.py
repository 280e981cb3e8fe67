"""Per-graph wavefront parity of the batched kernel (tw_decide_batch).

tw_solve_batch reports only treewidths and orderings; tw_decide_batch runs
decide(k) of many graphs through the same batched kernel and reports each
graph's level sizes and fingerprints, so the batch path is held to the same
bar as the single-graph path: every level of every run equal to the oracle's
(Section 3.1).  The graphs are the graphs with n <= 30 among the first 400
of the 4096-graph batch workload (185 graphs; the larger ones include runs of
10^9 states and more), at k = tw and k = tw - 1 (a yes run and a no run
each).
"""
import numpy as np
import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu

ORACLE_STATES = 400_000  # runs the oracle repeats here (a few seconds each)


def _rows(res, g):
    """Graph g's levels from the zero-padded rows: a yes run ends at its last
    non-empty level, a no run one level later, at its first empty level."""
    sizes = res["level_size"][g].tolist()
    last = max(i for i, x in enumerate(sizes) if x)
    if res["yes"][g] == 0:
        last += 1
    return sizes[: last + 1], res["fp_sum"][g][: last + 1].tolist(), res["fp_xor"][g][: last + 1].tolist()


@pytest.mark.parametrize("batch_kernel", [0, 1], ids=["persistent", "level_synchronous"])
def test_batch_levels_match_oracle_and_single_graph_path(batch_kernel):
    graphs = [a for a in gg.batch_graphs(400) if len(a) <= 30]
    with context(fingerprints=True, batch_kernel=batch_kernel) as ctx:
        sol = ctx.solve_batch(graphs, want_orders=False)
        assert np.all(sol["per_graph_status"] == 0)
        tw = sol["tw"]
        ks = np.concatenate([tw, np.maximum(tw - 1, 0)]).astype(np.int32)
        twice = graphs + graphs
        res = ctx.decide_batch(twice, ks)
        assert res["status"] == 0 and np.all(res["per_graph_status"] == 0)
        checked_oracle = 0
        for g, adj in enumerate(twice):
            k = int(ks[g])
            sizes, fs, fx = _rows(res, g)
            single = ctx.decide(adj, k=k)
            st = single["stats"]
            assert bool(res["yes"][g]) == single["yes"], (g, k)
            assert sizes == st["level_size"], (g, k)
            assert fs == st["fp_sum"] and fx == st["fp_xor"], (g, k)
            assert bool(res["yes"][g]) == (k >= int(tw[g % len(graphs)])), (g, k)
            if sum(sizes) <= ORACLE_STATES:
                exp = oracle.decide(adj, k)
                assert sizes == exp["level_size"], (g, k)
                assert fs == exp["fp_sum"] and fx == exp["fp_xor"], (g, k)
                checked_oracle += 1
        assert checked_oracle >= 150


@pytest.mark.parametrize("batch_kernel", [0, 1], ids=["persistent", "level_synchronous"])
def test_batch_levels_edge_cases(batch_kernel):
    # n > 64 (the single-graph path inside the batch call: the path P_70 at
    # k = 1, |L_i| = i + 1, and at k = 0, where L_1 is empty), k >= n-1 (the
    # single level {empty set}), an empty first level (K_7 at k = 2), n = 1
    graphs = [gg.path(70), gg.path(70), gg.complete(7), gg.workload_gnp20(), [0], gg.path(9)]
    ks = np.array([1, 0, 2, 25, 0, 1], np.int32)
    with context(fingerprints=True, batch_kernel=batch_kernel) as ctx:
        res = ctx.decide_batch(graphs, ks)
        assert res["status"] == 0
        for g, adj in enumerate(graphs):
            k = int(ks[g])
            sizes, fs, fx = _rows(res, g)
            if k >= len(adj) - 1:
                assert res["yes"][g] == 1 and sizes == [1] and fs == [0]
                continue
            exp = oracle.decide(adj, k)
            assert bool(res["yes"][g]) == exp["yes"], g
            assert sizes == exp["level_size"] and fs == exp["fp_sum"] and fx == exp["fp_xor"], g
        assert _rows(res, 0)[0] == list(range(1, 70))
        # a negative bound is refused for that graph only
        bad = ctx.decide_batch(graphs[:3], np.array([-1, 0, 2], np.int32))
        assert bad["per_graph_status"].tolist() == [1, 0, 0]


def test_persistent_batch_equals_level_synchronous_and_loop():
    # the same answers and verified orderings from the persistent kernel, the
    # level-synchronous kernel and a per-graph tw_solve loop, with proposed
    # bounds above, at and below tw
    graphs = [gg.mixed_graph(5000 + j, 12, 34, j % 2 == 0) for j in range(96)]
    with context() as ctx, context(batch_kernel=1) as sync:
        loop = [ctx.solve(a, want_order=False)["tw"] for a in graphs]
        for hint in (None, np.array(loop, np.float32) + 2, np.array(loop, np.float32) - 1):
            a = ctx.solve_batch(graphs, k_hint=hint)
            b = sync.solve_batch(graphs, k_hint=hint)
            assert a["status"] == 0 and b["status"] == 0
            assert a["tw"].tolist() == b["tw"].tolist() == loop
            pos = 0
            for g, adj in enumerate(graphs):
                order = a["orders"][pos: pos + len(adj)].tolist()
                assert sorted(order) == list(range(len(adj)))
                assert oracle.width_elim(adj, order) == loop[g]
                pos += len(adj)
    # graphs whose decide runs fit a block's arena never leave the persistent
    # kernel: the bounds and one launch for the whole batch (n <= 16: a run
    # holds fewer than 2^16 sets, the default arena)
    small = [gg.mixed_graph(6000 + j, 10, 16, j % 2 == 0) for j in range(200)]
    with context() as ctx, context(batch_kernel=1) as sync:
        a = ctx.solve_batch(small)
        b = sync.solve_batch(small)
    assert a["tw"].tolist() == b["tw"].tolist()
    assert a["stats"]["kernel_launches"] == 2 < b["stats"]["kernel_launches"]


def test_autotuned_persistent_batch_is_exact():
    # the first batch of >= 512 graphs picks 4 or 8 warps per block on a
    # sample; the answers do not depend on the choice
    graphs = [gg.mixed_graph(7000 + j, 10, 22, j % 2 == 0) for j in range(600)]
    with context(autotune=True) as tuned, context() as plain:
        a = tuned.solve_batch(graphs)
        b = plain.solve_batch(graphs)
        c2 = tuned.solve_batch(graphs[:50])  # the choice is kept for later batches
    assert a["status"] == 0 and b["status"] == 0 and c2["status"] == 0
    assert a["tw"].tolist() == b["tw"].tolist()
    assert c2["tw"].tolist() == b["tw"].tolist()[:50]
    pos = 0
    for g, adj in enumerate(graphs[:120]):
        order = a["orders"][pos: pos + len(adj)].tolist()
        assert oracle.width_elim(adj, order) == int(b["tw"][g])
        pos += len(adj)


@pytest.mark.parametrize("arena", [4096, 1 << 19])
def test_persistent_arena_size_does_not_change_answers(arena):
    # a small block arena sends most graphs on to the level-synchronous
    # kernel, a large one keeps them in the persistent kernel; the answers and
    # the orderings' widths are the same either way
    graphs = [gg.mixed_graph(8000 + j, 12, 30, j % 2 == 0) for j in range(120)]
    with context(batch_arena_states=arena) as ctx, context() as ref:
        a = ctx.solve_batch(graphs)
        b = ref.solve_batch(graphs)
    assert a["status"] == 0 and b["status"] == 0
    assert a["tw"].tolist() == b["tw"].tolist()
    pos = 0
    for g, adj in enumerate(graphs):
        order = a["orders"][pos: pos + len(adj)].tolist()
        assert oracle.width_elim(adj, order) == int(b["tw"][g])
        pos += len(adj)
