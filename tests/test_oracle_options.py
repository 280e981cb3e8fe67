"""Pins of the oracle's optional reductions (arXiv 1709.09990, Section 3.1:
maximum-clique skip and disjoint-path edges): same answers as the plain
method, valid orderings, and the helpers against brute force."""
import itertools
import math

import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg

OPTS = (oracle.CLIQUE_SKIP, oracle.DISJOINT_PATHS, oracle.CLIQUE_SKIP | oracle.DISJOINT_PATHS, oracle.MMW_PRUNE,
        oracle.CLIQUE_SKIP | oracle.DISJOINT_PATHS | oracle.MMW_PRUNE)


def _graphs(count, lo, hi, seed0):
    for s in range(count):
        rng = gg.Rng(seed0 + s)
        n = rng.randint(lo, hi)
        yield gg.gnp(n, 0.15 + 0.6 * rng.uniform(), seed0 + s, rng=rng)


@pytest.mark.parametrize("opts", OPTS)
def test_options_keep_every_answer(opts):
    for adj in _graphs(60, 2, 12, 7000):
        tw = oracle.solve(adj, want_order=False)["tw"]
        for k in range(max(0, tw - 2), min(len(adj), tw + 2)):
            d = oracle.decide_opts(adj, k, opts, want_order=True)
            assert d["yes"] == (k >= tw), (k, tw)
            if d["yes"]:
                assert oracle.width_q(adj, d["order"]) <= k


def _brute_max_clique(adj):
    n = len(adj)
    for size in range(n, 0, -1):
        for cand in itertools.combinations(range(n), size):  # lexicographic order
            if all((adj[a] >> b) & 1 for a, b in itertools.combinations(cand, 2)):
                return list(cand)
    return []


def test_max_clique_is_the_first_maximum():
    for adj in _graphs(80, 1, 11, 8000):
        assert oracle.max_clique(adj) == _brute_max_clique(adj)


def _brute_vertex_cut(adj, u, v):
    n = len(adj)
    others = [x for x in range(n) if x not in (u, v)]
    for size in range(len(others) + 1):
        for cut in itertools.combinations(others, size):
            blocked = set(cut)
            seen, stack = {u}, [u]
            while stack:
                x = stack.pop()
                for y in range(n):
                    if (adj[x] >> y) & 1 and y not in seen and y not in blocked:
                        seen.add(y)
                        stack.append(y)
            if v not in seen:
                return size
    return len(others)


def test_disjoint_paths_match_minimum_vertex_cuts():
    # Menger: internally disjoint u-v paths = smallest u-v vertex cut
    for adj in _graphs(40, 3, 9, 9000):
        n = len(adj)
        for u in range(n):
            for v in range(u + 1, n):
                if (adj[u] >> v) & 1:
                    continue
                assert oracle.disjoint_paths(adj, u, v, n) == _brute_vertex_cut(adj, u, v)


def test_closed_forms_with_clique_skip():
    # star K_{1,m}: the first maximum clique is {0, 1}; at k = 1 every subset
    # of the other m-1 leaves is feasible
    for m in range(3, 10):
        d = oracle.decide_opts(gg.star(m + 1), 1, oracle.CLIQUE_SKIP)
        assert d["yes"] and d["level_size"] == [math.comb(m - 1, i) for i in range(m)]
    # K_n: the clique is everything, so k < n-1 answers no at once
    for n in range(3, 8):
        d = oracle.decide_opts(gg.complete(n), n - 2, oracle.CLIQUE_SKIP)
        assert not d["yes"] and d["level_size"] == [1] and d["states_expanded"] == 0
    # K_{a,b} with a <= b: vertices on the b side have a disjoint paths
    g = gg.complete_bipartite(3, 5)
    assert oracle.disjoint_paths(g, 3, 4, 10) == 3 and oracle.disjoint_paths(g, 0, 1, 10) == 5


def _eliminated_graph(adj, S):
    """The graph left after eliminating the vertices of S one by one (each
    turns its neighbourhood into a clique), relabelled to 0..n-|S|-1."""
    n = len(adj)
    nb = {v: {u for u in range(n) if (adj[v] >> u) & 1} for v in range(n)}
    for v in range(n):
        if (S >> v) & 1:
            for a in nb[v]:
                nb[a].discard(v)
                nb[a] |= nb[v] - {a}
            del nb[v]
    keep = sorted(nb)
    pos = {v: i for i, v in enumerate(keep)}
    return [sum(1 << pos[u] for u in nb[v]) for v in keep]


def test_mmw_bound_is_a_lower_bound_of_the_remaining_graph():
    from oracle import bounds
    for adj in _graphs(60, 2, 10, 9500):
        n = len(adj)
        tw = oracle.brute_force_tw(adj)
        assert bounds.mmd_plus(adj) <= oracle.mmw_bound(adj, 0) <= tw
        rng = gg.Rng(n * 31 + 7)
        for _ in range(3):
            S = sum(1 << v for v in range(n) if rng.uniform() < 0.4)
            if bin(S).count("1") == n:
                continue
            H = _eliminated_graph(adj, S)
            assert oracle.mmw_bound(adj, S) <= oracle.brute_force_tw(H)


def test_mmw_bound_closed_forms():
    for n in range(2, 9):
        assert oracle.mmw_bound(gg.complete(n)) == n - 1
    for n in range(3, 10):
        assert oracle.mmw_bound(gg.cycle(n)) == 2
        assert oracle.mmw_bound(gg.path(n)) == 1
    # the second-smallest degree can exceed the smallest: a triangle with a
    # pendant vertex has degrees 1, 2, 2, 3 and tw 2
    g = [0b0110, 0b1101, 0b0011, 0b0010]
    assert oracle.mmw_bound(g) == 2
