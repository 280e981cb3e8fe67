"""The learned starting bound: exact answers always, fewer decide runs than
the plain sweep from the lower bound on held-out graphs."""
import numpy as np
import pytest

import oracle
from oracle import bounds as obounds
from paper_1709_09990_gb300 import graphgen as gg
from paper_1709_09990_gb300 import learned
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


def test_learned_bound_is_exact_and_saves_decide_runs():
    train_graphs = [gg.mixed_graph(10**6 + j, 12, 22, j % 2 == 0) for j in range(3000)]
    test_graphs = [gg.mixed_graph(2 * 10**6 + j, 16, 24, j % 2 == 0) for j in range(150)]
    with context(mem_cap_bytes=8 << 30) as ctx:
        L = learned.label(ctx, train_graphs)
        ok = L["status"] == 0
        assert ok.mean() > 0.95
        T = learned.train(ctx, L["x"][ok], L["tw"][ok], L["n"][ok], epochs=40)
        assert T["loss"][-1] < T["loss"][0]
        x = ctx.features(test_graphs)
        n = np.array([len(g) for g in test_graphs], np.int32)
        hint = learned.propose(ctx, T["params"], x, n, offset=-0.5)
        plain = ctx.solve_batch(test_graphs)
        hinted = ctx.solve_batch(test_graphs, k_hint=hint)
    assert plain["status"] == 0 and hinted["status"] == 0
    # exact: identical treewidths, every ordering verifies
    assert hinted["tw"].tolist() == plain["tw"].tolist()
    for g in range(0, len(test_graphs), 5):
        adj = test_graphs[g]
        if len(adj) > 20:
            continue
        lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
        assert oracle.solve(adj, k_start=lb, want_order=False)["tw"] == hinted["tw"][g]
    pos = 0
    for g, adj in enumerate(test_graphs):
        assert oracle.width_q(adj, hinted["orders"][pos: pos + len(adj)].tolist()) == hinted["tw"][g]
        pos += len(adj)
    # the gain: fewer decide runs than the sweep from the lower bound
    assert hinted["stats"]["decide_runs"] < plain["stats"]["decide_runs"]
