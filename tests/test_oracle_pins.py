"""Pins of the CPU oracle against facts that do not come from the oracle.

* brute force over all orderings with the explicit elimination game (the
  second characterisation in Section 2 of arXiv 1709.09990);
* an independent subset DP that tracks eliminated graphs explicitly;
* closed forms for treewidth and for level sizes of structured graphs;
* invariants of Q(S, v) and of the decision runs.
"""
import math

import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg


def small_graphs(count, n_lo=1, n_hi=9, seed0=0):
    out = []
    for s in range(count):
        rng = gg.Rng(seed0 + s)
        n = rng.randint(n_lo, n_hi)
        p = rng.uniform()
        out.append(gg.gnp(n, p, seed0 + s, rng=rng))
    return out


@pytest.mark.parametrize("block", range(4))
def test_tw_matches_brute_force(block):
    for adj in small_graphs(75, 1, 9, seed0=1000 * block):
        bf = oracle.brute_force_tw(adj)
        res = oracle.solve(adj, 0, want_order=True)
        assert res["tw"] == bf
        assert oracle.width_elim(adj, res["order"]) == bf
        assert oracle.width_q(adj, res["order"]) == bf


def test_brute_force_on_other_families():
    for s in range(20):
        for adj in (gg.rgg(9, 0.45, s), gg.partial_ktree(9, 3, s), gg.random_tree(9, s)):
            assert oracle.solve(adj)["tw"] == oracle.brute_force_tw(adj)


def test_width_q_equals_elimination_game():
    # Q(prefix(v), v) is the neighbourhood of v in the eliminated graph, so
    # both widths agree on every ordering, not only on optimal ones.
    for s in range(60):
        adj = gg.gnp(12, 0.35, 500 + s)
        order = gg.relabel(list(range(12)), s)  # just a permutation source
        perm = list(range(12))
        rng = gg.Rng(s)
        for i in range(11, 0, -1):
            j = rng.randint(0, i)
            perm[i], perm[j] = perm[j], perm[i]
        assert oracle.width_q(adj, perm) == oracle.width_elim(adj, perm)


def _check_levels_vs_subset_dp(adj, k):
    a = oracle.decide(adj, k)
    b = oracle.subset_dp(adj, k)
    assert a["yes"] == b["yes"]
    assert a["levels"] == b["levels"]
    assert a["level_size"] == b["level_size"]
    assert a["fp_sum"] == b["fp_sum"]
    assert a["fp_xor"] == b["fp_xor"]


@pytest.mark.parametrize("block", range(3))
def test_levels_match_subset_dp(block):
    for s in range(25):
        rng = gg.Rng(77 + 100 * block + s)
        n = rng.randint(2, 14)
        adj = gg.gnp(n, 0.15 + 0.5 * rng.uniform(), 77 + 100 * block + s, rng=rng)
        tw = oracle.solve(adj, want_order=False)["tw"]
        for k in {max(0, tw - 2), max(0, tw - 1), tw, tw + 1}:
            _check_levels_vs_subset_dp(adj, k)


def test_levels_match_subset_dp_gnp20():
    adj = gg.workload_gnp20()
    for k in (6, 7, 8):
        _check_levels_vs_subset_dp(adj, k)


def test_closed_form_treewidths():
    for n in range(1, 9):
        assert oracle.solve(gg.complete(n))["tw"] == n - 1
        assert oracle.solve([0] * n)["tw"] == 0
    for n in range(2, 14):
        assert oracle.solve(gg.random_tree(n, n))["tw"] == 1
        assert oracle.solve(gg.path(n))["tw"] == 1
    for n in range(3, 14):
        assert oracle.solve(gg.cycle(n))["tw"] == 2
    for a, b in [(2, 2), (2, 5), (3, 3), (3, 4), (3, 5), (4, 4)]:
        assert oracle.solve(gg.grid(a, b))["tw"] == min(a, b)
    for a, b in [(1, 4), (2, 3), (3, 4), (4, 4), (2, 7)]:
        assert oracle.solve(gg.complete_bipartite(a, b))["tw"] == min(a, b)
    for k in range(1, 5):
        for s in range(3):
            assert oracle.solve(gg.ktree(k + 6, k, s))["tw"] == k
            assert oracle.solve(gg.partial_ktree(k + 8, k, s))["tw"] <= k


def test_closed_form_level_sizes():
    for n in range(2, 12):
        d = oracle.decide([0] * n, 0)
        assert d["level_size"] == [math.comb(n, i) for i in range(n)]
        d = oracle.decide(gg.path(n), 1)
        assert d["level_size"] == [i + 1 for i in range(n - 1)]
        d = oracle.decide(gg.star(n), 1)
        assert d["level_size"] == [math.comb(n - 1, i) for i in range(n - 1)]
    for n in range(3, 12):
        d = oracle.decide(gg.cycle(n), 2)
        assert d["level_size"] == [math.comb(n, i) for i in range(n - 2)]
    for n in range(3, 9):
        for k in range(0, n - 1):
            d = oracle.decide(gg.complete(n), k)
            assert d["level_size"] == [1, 0] and not d["yes"]


def test_trivial_bounds_and_degenerate_inputs():
    d = oracle.decide([0], 0)
    assert d["yes"] and d["level_size"] == [1] and d["states_expanded"] == 0
    assert oracle.solve([0])["order"] == [0]
    adj = gg.gnp(7, 0.5, 3)
    d = oracle.decide(adj, 6)  # k >= n-1: the level loop is empty
    assert d["yes"] and d["levels"] == 1
    with pytest.raises(ValueError):
        oracle.decide(adj, -1)


def test_q_set_invariants():
    for s in range(30):
        adj = gg.gnp(14, 0.3, 900 + s)
        rng = gg.Rng(s)
        S = 0
        for v in range(14):
            if rng.uniform() < 0.5:
                S |= 1 << v
        for v in range(14):
            q = oracle.q_set(adj, S, v)
            assert q & S == 0 and not (q >> v) & 1
            assert bin(q).count("1") == oracle.q_size(adj, S, v)
            # with S empty Q is the neighbourhood
            assert oracle.q_set(adj, 0, v) == adj[v]


def test_monotone_in_k_and_counters():
    for s in range(15):
        adj = gg.gnp(11, 0.4, 300 + s)
        ans = [oracle.decide(adj, k)["yes"] for k in range(11)]
        first = ans.index(True)
        assert all(ans[first:]) and not any(ans[:first])
        d = oracle.decide(adj, first)
        n = len(adj)
        assert d["states_expanded"] == sum(d["level_size"][:-1])
        assert d["candidates"] == sum(sz * (n - i) for i, sz in enumerate(d["level_size"][:-1]))
        assert d["feasible"] >= d["level_size"][-1]


def test_tw_invariant_under_relabelling():
    for s in range(20):
        adj = gg.gnp(10, 0.35, 40 + s)
        assert oracle.solve(adj)["tw"] == oracle.solve(gg.relabel(adj, s))["tw"]


def test_fingerprint_is_splitmix64_output():
    # the first output of splitmix64 from seed 0 (Steele, Lea & Flood 2014)
    # is the output function applied to the golden-ratio increment
    assert oracle.fingerprint(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_fingerprint_distinguishes_words():
    assert oracle.fingerprint(1) != oracle.fingerprint(1 << 64)
    assert oracle.fingerprint(0) == 0


def test_decide_prefix_is_the_start_of_decide():
    # the truncated run builds exactly the first levels of the full run
    from paper_1709_09990_gb300 import graphgen as gg
    for adj, k in ((gg.workload_gnp20(), 8), (gg.gnp(14, 0.4, 7), 5), (gg.partial_ktree(16, 4, 1), 4)):
        full = oracle.decide(adj, k, count_canonical=True)
        for m in range(0, full["levels"]):
            p = oracle.decide_prefix(adj, k, m)
            assert p["levels"] == min(m + 1, full["levels"])
            for key in ("level_size", "fp_sum", "fp_xor"):
                assert p[key] == full[key][: p["levels"]], (k, m, key)
        last = oracle.decide_prefix(adj, k, full["levels"])
        for key in ("states_expanded", "candidates", "feasible", "canonical"):
            assert last[key] == full[key], key
