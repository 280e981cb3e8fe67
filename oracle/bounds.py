"""Treewidth bounds and graph features, plain Python (test infrastructure).

Only tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  Vertex sets are Python ``set`` objects; nothing is vectorised.

Lower bounds:
  * ``mmd`` - minimum degree of the graph, maximised while a minimum-degree
    vertex is deleted repeatedly (degeneracy).
  * ``mmd_plus`` - minor-min-width, also called MMD+(min-d) (arXiv 1709.09990,
    Section 3.3): repeatedly take a minimum-degree vertex v, record its degree,
    and contract it into its minimum-degree neighbour u (v disappears, u keeps
    N(u) u N(v) minus u and v); an isolated v is deleted.  The largest degree
    recorded is a lower bound because minors do not increase treewidth.
Upper bounds (widths of greedy elimination orderings):
  * ``min_degree_ub`` - eliminate a minimum-degree vertex each step.
  * ``min_fill_ub`` - eliminate the vertex whose neighbourhood misses the
    fewest edges each step.
Ties always go to the lowest vertex index.  ``mmd_plus_steps``,
``min_degree_order`` and ``min_fill_order`` return the choices themselves, so
that tests can pin every selection rule on hand-worked graphs.

Features (12, the input of the learned starting bound), with d(v) the degree:
  0 n/64; 1 edge density 2|E|/(n(n-1)); 2 min d / n; 3 max d / n;
  4 mean d / n; 5 population std of d / n; 6-9 fraction of vertices with
  d/n in [0,.25), [.25,.5), [.5,.75), [.75,1]; 10 mmd_plus / n;
  11 (min_degree_ub + min_fill_ub) / (2n).
"""

from __future__ import annotations

import math
from typing import Dict, List, Sequence, Set


def _adjsets(adj: Sequence[int]) -> Dict[int, Set[int]]:
    n = len(adj)
    return {v: {u for u in range(n) if (adj[v] >> u) & 1} for v in range(n)}


def _argmin_degree(g: Dict[int, Set[int]], among=None) -> int:
    cands = sorted(g) if among is None else sorted(among)
    best = cands[0]
    for v in cands[1:]:
        if len(g[v]) < len(g[best]):
            best = v
    return best


def mmd(adj: Sequence[int]) -> int:
    g = _adjsets(adj)
    lb = 0
    while g:
        v = _argmin_degree(g)
        lb = max(lb, len(g[v]))
        for u in g[v]:
            g[u].discard(v)
        del g[v]
    return lb


def mmd_plus_steps(adj: Sequence[int]) -> List[tuple]:
    """The contraction sequence of ``mmd_plus``: one (v, degree of v, u) per
    step, u = the neighbour v is contracted into (None when v is isolated and
    simply deleted)."""
    g = _adjsets(adj)
    steps = []
    while len(g) >= 2:
        v = _argmin_degree(g)
        d = len(g[v])
        if not g[v]:
            del g[v]
            steps.append((v, 0, None))
            continue
        u = _argmin_degree(g, g[v])
        # contract v into u
        for w in g[v]:
            g[w].discard(v)
            if w != u:
                g[w].add(u)
                g[u].add(w)
        del g[v]
        steps.append((v, d, u))
    return steps


def mmd_plus(adj: Sequence[int]) -> int:
    return max([d for _, d, _ in mmd_plus_steps(adj)] + [0])


def _eliminate(g: Dict[int, Set[int]], v: int) -> int:
    nb = g[v]
    for a in nb:
        g[a].discard(v)
        for b in nb:
            if a != b:
                g[a].add(b)
    del g[v]
    return len(nb)


def width_of_order(adj: Sequence[int], order: Sequence[int]) -> int:
    """Largest degree met when the vertices are eliminated in this order."""
    g = _adjsets(adj)
    return max([_eliminate(g, v) for v in order] + [0])


def min_degree_order(adj: Sequence[int]) -> List[int]:
    """Greedy ordering: eliminate a minimum-degree vertex of the current graph."""
    g = _adjsets(adj)
    order = []
    while g:
        v = _argmin_degree(g)
        order.append(v)
        _eliminate(g, v)
    return order


def min_degree_ub(adj: Sequence[int]) -> int:
    return width_of_order(adj, min_degree_order(adj))


def _fill(g: Dict[int, Set[int]], v: int) -> int:
    nb = sorted(g[v])
    missing = 0
    for i, a in enumerate(nb):
        for b in nb[i + 1:]:
            if b not in g[a]:
                missing += 1
    return missing


def min_fill_order(adj: Sequence[int]) -> List[int]:
    """Greedy ordering: eliminate the vertex whose neighbourhood misses the
    fewest edges in the current graph."""
    g = _adjsets(adj)
    order = []
    while g:
        cands = sorted(g)
        best = cands[0]
        best_fill = _fill(g, best)
        for v in cands[1:]:
            f = _fill(g, v)
            if f < best_fill:
                best, best_fill = v, f
        order.append(best)
        _eliminate(g, best)
    return order


def min_fill_ub(adj: Sequence[int]) -> int:
    return width_of_order(adj, min_fill_order(adj))


def features(adj: Sequence[int]) -> List[float]:
    n = len(adj)
    deg = [bin(r).count("1") for r in adj]
    m = sum(deg) // 2
    density = (2.0 * m / (n * (n - 1))) if n > 1 else 0.0
    mean = sum(deg) / n
    var = sum((d - mean) ** 2 for d in deg) / n
    hist = [0, 0, 0, 0]
    for d in deg:
        # bin edges compared in integers: d/n < 1/4, < 1/2, < 3/4
        b = 0 if 4 * d < n else 1 if 2 * d < n else 2 if 4 * d < 3 * n else 3
        hist[b] += 1
    return [n / 64.0, density, min(deg) / n, max(deg) / n, mean / n, math.sqrt(var) / n,
            hist[0] / n, hist[1] / n, hist[2] / n, hist[3] / n,
            mmd_plus(adj) / n, (min_degree_ub(adj) + min_fill_ub(adj)) / (2.0 * n)]
