"""GPU decide/solve with the optional reductions of Section 3.1 against the
oracle with the same options: answers, level sizes, fingerprints, counters."""
import numpy as np
import pytest

import oracle
from oracle import bounds as obounds
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu

OPTS = {"clique": (True, False, False, oracle.CLIQUE_SKIP), "paths": (False, True, False, oracle.DISJOINT_PATHS),
        "both": (True, True, False, oracle.CLIQUE_SKIP | oracle.DISJOINT_PATHS),
        "mmw": (False, False, True, oracle.MMW_PRUNE),
        "all": (True, True, True, oracle.CLIQUE_SKIP | oracle.DISJOINT_PATHS | oracle.MMW_PRUNE)}


def _check(ctx, adj, k, o):
    exp = oracle.decide_opts(adj, k, o | oracle.COUNT_CANONICAL)
    got = ctx.decide(adj, k=k, want_order=True)
    st = got["stats"]
    assert got["yes"] == exp["yes"]
    for key in ("level_size", "fp_sum", "fp_xor", "states_expanded", "candidates"):
        assert st[key] == exp[key], (k, key)
    # with minor-min-width pruning every feasible pair is submitted, else only
    # the canonical ones
    assert st["generated"] == exp["feasible" if o & oracle.MMW_PRUNE else "canonical"], k
    if got["yes"]:
        assert oracle.width_q(adj, got["order"].tolist()) <= k


@pytest.mark.parametrize("name", sorted(OPTS))
@pytest.mark.parametrize("graph_levels", [-1, 1])
def test_options_match_oracle(name, graph_levels):
    cs, dp, mm, o = OPTS[name]
    # (dense graphs make the oracle's exhaustive clique search slow; the
    # 128-bit states are covered by a relabelled path on 70 vertices)
    graphs = [gg.workload_gnp20(), gg.gnp(44, 0.5, 4), gg.relabel(gg.path(70), 5), gg.partial_ktree(26, 5, 3)]
    graphs += [gg.gnp(14 + s, 0.35, 4000 + s) for s in range(6)]
    with context(fingerprints=True, clique_skip=cs, disjoint_paths=dp, mmw_prune=mm, graph_levels=graph_levels) as ctx:
        for adj in graphs:
            lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
            tw = oracle.solve(adj, k_start=lb, want_order=False)["tw"]
            for k in (tw - 1, tw):
                _check(ctx, adj, k, o)
                _check(ctx, adj, k, o)  # again, over the buffers the first call left


@pytest.mark.parametrize("name", sorted(OPTS))
def test_solve_with_options_is_exact(name):
    cs, dp, mm, _ = OPTS[name]
    with context(clique_skip=cs, disjoint_paths=dp, mmw_prune=mm) as ctx:
        for s in range(8):
            adj = gg.mixed_graph(6000 + s, 10, 26, s % 2 == 0)
            tw = oracle.solve(adj, want_order=False)["tw"] if len(adj) <= 18 else None
            sol = ctx.solve(adj, want_order=True, want_td=True)
            plain = None
            if tw is None:
                with context() as p:
                    plain = p.solve(adj)["tw"]
            assert sol["tw"] == (tw if tw is not None else plain)
            assert oracle.width_q(adj, sol["order"].tolist()) == sol["tw"]
            assert oracle.verify_td(adj, sol["td_parent"], sol["td_bags"]) == sol["tw"]
