"""The pins catch plausible mistakes: each mutant below is the oracle with one
planted error (a dropped statement, an off-by-one bound, a swapped branch, a
wrong index); it is compiled on the CPU and must fail at least one pin."""
import ctypes
import math
import os
import subprocess

import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg
from tests.test_oracle_canonical import _levels

SRC = os.path.join(os.path.dirname(oracle.__file__), "tw_oracle.cpp")

MUTANTS = {
    "v_in_its_own_q": ("return without(set_minus(ends, S), v);", "return set_minus(ends, S);"),
    "q_misses_direct_neighbours": ("const Key ends = set_union(g.nset[v], neighbours_of(g, inner));",
                                   "const Key ends = neighbours_of(g, inner);"),
    "reach_stops_after_one_step": ("  while (!is_empty(newest)) {\n    newest = set_minus(",
                                   "  while (!is_empty(newest) && false) {\n    newest = set_minus("),
    "reach_leaves_s": ("newest = set_minus(set_meet(neighbours_of(g, newest), inside), reached);",
                       "newest = set_minus(set_minus(neighbours_of(g, newest), inside), reached);"),
    "strict_degree_bound": ("if (q_size(g, S, v) > k) continue;", "if (q_size(g, S, v) >= k) continue;"),
    "one_level_short": ("const int top = n - k - 1;", "const int top = n - k - 2;"),
    "wrong_vertex_added": ("next.emplace(with(S, v), v);", "next.emplace(with(S, (v + 1) % g.n), v);"),
    "fill_in_self_loop": ("if ((nb >> u) & 1u) r |= nb & ~(1u << u);", "if ((nb >> u) & 1u) r |= nb;"),
    "width_off_by_one": ("width = std::max(width, (int)nb.size());", "width = std::max(width, (int)nb.size() - 1);"),
    "no_stop_at_empty_level": ("while ((int)L.size() - 1 < stop && !L.back().empty()) {",
                               "while ((int)L.size() - 1 < stop) {"),
    "fingerprint_constant": ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 27)) * 0x94D049BB133111EDULL;"),
    "canonical_highest_vertex": ("const int low = lowest_vertex(T);",
                                 "const int low = T.w[1] ? 127 - __builtin_clzll(T.w[1]) : 63 - __builtin_clzll(T.w[0]);"),
    "canonical_search_leaves_set": ("return low == v || has(reach_within(g, T, v), low);",
                                    "return low == v || has(reach_within(g, Key{{~0ULL, ~0ULL}}, v), low);"),
    "prefix_one_level_short": ("std::min(top, max_level) : top;", "std::min(top, max_level - 1) : top;"),
}


def _pins_hold() -> bool:
    try:
        for s in range(40):
            rng = gg.Rng(31 + s)
            n = rng.randint(2, 7)
            adj = gg.gnp(n, 0.2 + 0.6 * rng.uniform(), 31 + s, rng=rng)
            res = oracle.solve(adj)
            assert res["tw"] == oracle.brute_force_tw(adj)
            assert oracle.width_elim(adj, res["order"]) == res["tw"]
        for s in range(8):
            adj = gg.gnp(10, 0.35, 500 + s)
            tw = oracle.solve(adj, want_order=False)["tw"]
            for k in (max(0, tw - 1), tw):
                a, b = oracle.decide(adj, k), oracle.subset_dp(adj, k)
                assert (a["yes"], a["level_size"], a["fp_sum"]) == (b["yes"], b["level_size"], b["fp_sum"])
        assert oracle.solve(gg.cycle(7))["tw"] == 2
        assert oracle.decide(gg.path(8), 1)["level_size"] == [i + 1 for i in range(7)]
        assert oracle.decide([0] * 6, 0)["level_size"] == [math.comb(6, i) for i in range(6)]
        for s in range(12):
            rng = gg.Rng(700 + s)
            n = rng.randint(3, 7)
            adj = gg.gnp(n, 0.2 + 0.6 * rng.uniform(), 700 + s, rng=rng)
            for k in range(n):
                assert oracle.decide(adj, k, count_canonical=True)["canonical"] == _levels(adj, k, True)[1]
        assert oracle.decide([0] * 6, 0, count_canonical=True)["canonical"] == 2 ** 6 - 2
        adj = gg.gnp(12, 0.3, 77)
        full = oracle.decide(adj, 3)
        for m in (1, 4):
            assert oracle.decide_prefix(adj, 3, m)["level_size"] == full["level_size"][: m + 1]
        # splitmix64's first output from seed 0 (Steele, Lea & Flood 2014)
        assert oracle.fingerprint(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
        return True
    except AssertionError:
        return False


def test_unmutated_oracle_passes_the_quick_pins():
    assert _pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    mutated = src.replace(old, new, 1)
    cpp = tmp_path / f"{name}.cpp"
    so = tmp_path / f"lib_{name}.so"
    cpp.write_text(mutated)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(cpp)])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(str(so))))
    assert not _pins_hold(), f"mutant {name} passed every pin"
