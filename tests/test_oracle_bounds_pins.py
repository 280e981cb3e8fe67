"""Hand-worked pins of the selection rules in ``oracle/bounds.py``.

Every lower or upper bound stays valid whichever minimum-degree vertex,
contraction partner or minimum-fill vertex is chosen, so inequalities alone
(MMD <= MMD+ <= tw <= the greedy widths) cannot fix the rules the GPU's
``bounds_kernel`` is compared with.  The graphs below are small enough to
follow by hand, and each one is chosen so that a different rule gives a
different value:

* MMD+ (minor-min-width, Section 3.3): a minimum-degree vertex v (lowest index
  on ties) is contracted into its minimum-degree neighbour (lowest index).
* min-degree width: eliminate a minimum-degree vertex, lowest index on ties.
* min-fill width: eliminate the vertex whose neighbourhood misses the fewest
  edges, lowest index on ties.

The mutation check at the end plants the plausible mistakes (the maximum-
degree neighbour, the highest index on ties, the fill counted with the wrong
sign, a shifted histogram bin edge) in copies of the module and requires each
to fail one of these pins.
"""
import math
import os
import types

import pytest

import oracle
from oracle import bounds
from paper_1709_09990_gb300 import graphgen as gg


def _graph(nbrs):
    """Adjacency bitmasks from neighbour lists (checked to be symmetric)."""
    adj = [0] * len(nbrs)
    for v, ns in enumerate(nbrs):
        for u in ns:
            assert v in nbrs[u], (v, u)
            adj[v] |= 1 << u
    return adj


# B1.  Degrees 4, 3, 4, 4, 3, 4.  Vertex 1 (degree 3, lower index than 4) has
# neighbours 2, 3, 4 of degrees 4, 4, 3, so it is contracted into 4; 4 then
# gains 2 and 3, and {0, 2, 3, 4, 5} is a K5: the next step records degree 4.
# Contracting 1 into a maximum-degree neighbour (2) instead leaves vertices of
# degree 3, and that rule ends with 3.
B1 = _graph([[2, 3, 4, 5], [2, 3, 4], [0, 1, 3, 5], [0, 1, 2, 5], [0, 1, 5], [0, 2, 3, 4]])
B1_STEPS = [(1, 3, 4), (0, 4, 2), (2, 3, 3), (3, 2, 4), (4, 1, 5)]

# B2.  K_{3,3} between {0, 1, 2} and {3, 4, 5} plus the edge 12.  Vertices 0,
# 3, 4, 5 tie at degree 3; eliminating 0 (lowest index) makes {3, 4, 5} a
# triangle, and the five vertices left form a K5: width 4.  Taking 5 first
# (highest index) keeps the width at 3, the treewidth.
B2 = _graph([[3, 4, 5], [2, 3, 4, 5], [1, 3, 4, 5], [0, 1, 2], [0, 1, 2], [0, 1, 2]])

# B3.  Degrees 3, 4, 3, 4, 3, 3, 4.  Lowest index first: 0 goes into 2 (its
# neighbours 2, 3, 5 have degrees 3, 4, 3), then 2 into 3, then 4 into 1,
# which leaves the K4 {1, 3, 5, 6}: every recorded degree is at most 3.  With
# the highest index first the sequence starts at 5 and records a degree 4.
B3 = _graph([[2, 3, 5], [3, 4, 5, 6], [0, 3, 4], [0, 1, 2, 6], [1, 2, 6], [0, 1, 6], [1, 3, 4, 5]])
B3_STEPS = [(0, 3, 2), (2, 3, 3), (4, 3, 1), (1, 3, 3), (3, 2, 5), (5, 1, 6)]

# B4.  Every vertex misses exactly 3 edges in its neighbourhood (for 0:
# 25, 35, 56), so the tie rule alone picks the first vertex.  Eliminating 0
# (degree 4) adds 25, 35, 56; then 1 misses nothing, and {2, .., 6} is a K5:
# width 4.  Eliminating 6 first (degree 5) already gives width 5.
B4 = _graph([[2, 3, 5, 6], [2, 3, 5, 6], [0, 1, 3, 4, 6], [0, 1, 2, 4, 6], [2, 3, 5, 6], [0, 1, 4],
             [0, 1, 2, 3, 4]])

# B5.  The path 0-1-2 plus an isolated vertex 3: 0 misses no edge and 1
# misses 02, so minimum fill eliminates 0 first (width 1); maximum fill would
# start with 1 (degree 2).
B5 = _graph([[1], [0, 2], [1], []])


def _fill_of(adj, v):
    ns = [u for u in range(len(adj)) if (adj[v] >> u) & 1]
    return sum(1 for i, a in enumerate(ns) for b in ns[i + 1:] if not (adj[a] >> b) & 1)


def _check_pins(b) -> None:
    """The pins, against a bounds module b (the real one or a mutant)."""
    assert b.mmd_plus_steps(B1) == B1_STEPS
    assert b.mmd_plus(B1) == 4
    assert b.min_degree_order(B2) == [0, 1, 2, 3, 4, 5]
    assert b.min_degree_ub(B2) == 4
    assert b.mmd(B2) == 3
    assert b.mmd_plus_steps(B3) == B3_STEPS
    assert b.mmd_plus(B3) == 3
    assert all(_fill_of(B4, v) == 3 for v in range(7))
    assert b.min_fill_order(B4)[:2] == [0, 1]
    assert b.min_fill_ub(B4) == 4
    assert b.min_fill_order(B5)[0] == 0 and b.min_fill_ub(B5) == 1
    # degree histogram bin edges: in C_8 every degree is 2 = n/4, which lies in
    # [.25, .5); in K_{1,3} the leaves have degree 1 < 4/4 and the centre 3
    f = b.features(gg.cycle(8))
    assert f[6:10] == [0.0, 1.0, 0.0, 0.0]
    f = b.features(gg.star(4))
    assert f[6:10] == [0.0, 0.75, 0.0, 0.25]


def test_hand_worked_selection_rules():
    _check_pins(bounds)


def test_hand_worked_graphs_against_brute_force():
    # the bounds bracket the exact treewidth of each hand-worked graph
    assert oracle.brute_force_tw(B1) == 4  # the K5 minor and a width-4 ordering
    assert oracle.brute_force_tw(B2) == 3  # K_{3,3} has treewidth 3
    for adj in (B1, B2, B3, B4, B5):
        tw = oracle.brute_force_tw(adj)
        assert bounds.mmd(adj) <= bounds.mmd_plus(adj) <= tw <= min(bounds.min_degree_ub(adj),
                                                                    bounds.min_fill_ub(adj))
        assert bounds.width_of_order(adj, bounds.min_degree_order(adj)) == oracle.width_elim(
            adj, bounds.min_degree_order(adj))


MUTANTS = {
    "mmd_plus_max_degree_neighbour": ("        u = _argmin_degree(g, g[v])\n",
                                      "        u = max(sorted(g[v]), key=lambda x: len(g[x]))\n"),
    "mmd_plus_highest_index": ("    while len(g) >= 2:\n        v = _argmin_degree(g)\n",
                               "    while len(g) >= 2:\n        v = min(sorted(g, reverse=True), key=lambda x: len(g[x]))\n"),
    "min_degree_highest_index": ("    while g:\n        v = _argmin_degree(g)\n        order.append(v)\n",
                                 "    while g:\n        v = min(sorted(g, reverse=True), key=lambda x: len(g[x]))\n"
                                 "        order.append(v)\n"),
    "min_fill_wrong_sign": ("            if f < best_fill:\n", "            if f > best_fill:\n"),
    "min_fill_highest_index": ("        cands = sorted(g)\n", "        cands = sorted(g, reverse=True)\n"),
    "histogram_edge_inclusive": ("b = 0 if 4 * d < n else", "b = 0 if 4 * d <= n else"),
}


def _load_mutant(name, old, new):
    src = open(bounds.__file__).read()
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    mod = types.ModuleType(f"bounds_{name}")
    exec(compile(src.replace(old, new), f"<bounds mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_bounds_mutant_fails_a_pin(name):
    mod = _load_mutant(name, *MUTANTS[name])
    with pytest.raises(AssertionError):
        _check_pins(mod)
