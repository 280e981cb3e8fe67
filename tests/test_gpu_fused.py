"""The fused small solve: the whole k sweep, walk and tree decomposition of a
graph with n <= 64 in one cooperative launch (Section 3.1's iterative
deepening of Listing 1, grid barriers between levels).

Checked against the oracle: treewidth, the level sizes and fingerprints of
the final decide run, verified orderings and tree decompositions; the path
that gives up (an arena too small for the levels) must hand over to the level
loop without changing any result; and the launch count shows the sweep runs
in one launch.  The sweep's decide runs k, k+1, k+2 run at the same time in
separate groups of blocks; the answer and counters must be those of the
sequential sweep.
"""
import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


def _graphs():
    out = [("gnp20", gg.workload_gnp20()), ("path9", gg.path(9)), ("k7", gg.complete(7)), ("edgeless5", [0] * 5),
           ("single", [0]), ("grid4x5", gg.grid(4, 5)), ("pktree26", gg.partial_ktree(26, 3, 3)),
           ("path60", gg.path(60)), ("gnp44", gg.gnp(44, 0.5, 4))]
    for s in range(6):
        rng = gg.Rng(4000 + s)
        n = rng.randint(8, 24)
        out.append((f"gnp{n}_{s}", gg.gnp(n, 0.2 + 0.5 * rng.uniform(), 4000 + s, rng=rng)))
    return out


@pytest.mark.parametrize("name,adj", _graphs(), ids=[n for n, _ in _graphs()])
def test_fused_solve_matches_oracle(name, adj):
    ref = oracle.solve(adj, k_start=_lb(adj), want_order=False)
    exp = oracle.decide(adj, ref["tw"])
    with context(fingerprints=True) as ctx:
        sol = ctx.solve(adj, want_order=True, want_td=True)
    assert sol["tw"] == ref["tw"]
    order = sol["order"].tolist()
    assert sorted(order) == list(range(len(adj)))
    assert oracle.width_q(adj, order) == ref["tw"]
    assert oracle.verify_td(adj, sol["td_parent"], sol["td_bags"]) == ref["tw"]
    st = sol["stats"]
    assert st["level_size"] == exp["level_size"]
    assert st["fp_sum"] == exp["fp_sum"] and st["fp_xor"] == exp["fp_xor"]


@pytest.mark.parametrize("name,adj,tw", [("gnp20", gg.workload_gnp20(), 8), ("pktree26", gg.partial_ktree(26, 3, 3), None),
                                         ("gnp44", gg.gnp(44, 0.5, 4), None), ("path9", gg.path(9), 1)])
def test_fused_solve_is_one_launch_and_counts_like_the_loop(name, adj, tw):
    # decide runs k, k+1, k+2 of the sweep run at once, one per group of
    # blocks; the runs above the answer are speculative and not counted, so
    # the counters are those of the sequential level loop whether tw is the
    # lower bound (pktree26, path9), two above it (gnp20) or many windows of
    # three runs away (gnp44)
    with context() as fused, context(fused_states=-1) as loop:
        a = fused.solve(adj, want_td=True)
        b = loop.solve(adj, want_td=True)
    assert a["tw"] == b["tw"]
    if tw is not None:
        assert a["tw"] == tw
    for key in ("states_expanded", "candidates", "generated", "decide_runs", "level_size"):
        assert a["stats"][key] == b["stats"][key], key
    # bounds + the fused solve
    assert a["stats"]["kernel_launches"] <= 3 < b["stats"]["kernel_launches"]


@pytest.mark.parametrize("cap", [64, 3000])
def test_fused_solve_that_gives_up_hands_over(cap):
    # an arena of 64 or 3000 states: the fused run gives up at the first k (or
    # a later one) and the level loop finishes the sweep from there
    for adj in (gg.workload_gnp20(), gg.gnp(44, 0.5, 4)):
        ref = oracle.solve(adj, k_start=_lb(adj), want_order=False)
        with context(fingerprints=True, fused_states=cap) as ctx:
            sol = ctx.solve(adj, want_order=True, want_td=True)
            again = ctx.solve(adj, want_order=True)  # remembered: no second fused attempt
        assert sol["tw"] == again["tw"] == ref["tw"]
        assert oracle.width_elim(adj, sol["order"].tolist()) == ref["tw"]
        assert oracle.verify_td(adj, sol["td_parent"], sol["td_bags"]) == ref["tw"]
        exp = oracle.decide(adj, ref["tw"])
        assert sol["stats"]["level_size"] == exp["level_size"] and sol["stats"]["fp_sum"] == exp["fp_sum"]
        assert again["stats"]["states_expanded"] == oracle.solve(adj, k_start=_lb(adj),
                                                                  want_order=False)["states_expanded"]


def _lb(adj):
    from oracle import bounds
    return max(bounds.mmd(adj), bounds.mmd_plus(adj))


def test_fused_decide_matches_oracle():
    adj = gg.workload_gnp20()
    with context(fingerprints=True) as ctx:
        for k in (5, 7, 8, 19, 25):
            got = ctx.decide(adj, k=k, want_order=True)
            exp = oracle.decide(adj, k)
            assert got["yes"] == exp["yes"], k
            assert got["stats"]["level_size"] == exp["level_size"], k
            assert got["stats"]["fp_sum"] == exp["fp_sum"], k
            assert got["stats"]["states_expanded"] == exp["states_expanded"], k
            if got["yes"]:
                assert oracle.width_q(adj, got["order"].tolist()) <= k
