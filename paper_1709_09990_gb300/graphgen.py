"""Seeded synthetic graph generators.

This module is input generation only: it draws random graphs and holds none
of the treewidth method's arithmetic.  Both the CPU oracle (``oracle/``) and
the CUDA path are fed from it, so that the two sides see identical inputs.

Random source: splitmix64 (Steele, Lea & Flood, 2014) expands a 64-bit seed
into the 256-bit state of xoshiro256** (Blackman & Vigna, 2018).  A uniform
double in [0, 1) is the top 53 bits of a draw times 2^-53, and an integer
uniform on {a..b} is ``a + floor(u * (b - a + 1))``.

Graphs are returned as a list of Python ints, one adjacency bitmask per
vertex (bit j of row i set iff ij is an edge), which converts losslessly to
the uint32 / uint64 row layouts of the C ABI with :func:`to_rows_u64` and
:func:`to_rows_u32`.

Families (the paper evaluates on external benchmark instances that are not
available here; these seeded families stand in for them):

* ``gnp(n, p, seed)``: Erdos-Renyi; the pairs i<j are visited in
  lexicographic order and ij is an edge iff the next uniform draw is < p.
* ``rgg(n, r, seed)``: random geometric graph; n points (x, y) are drawn in
  vertex order (x first), and ij is an edge iff the squared distance is
  <= r^2.
* ``ktree(n, k, seed)``: random k-tree; starts from K_{k+1} and attaches each
  new vertex to a uniformly chosen k-clique of the clique list.
* ``partial_ktree(n, k, seed, remove_frac=0.3)``: a random k-tree with
  floor(remove_frac*|E| + 1/2) of its edges removed, chosen by a Fisher-Yates
  shuffle of the lexicographic edge list (the same random stream continues).
"""

from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

MASK64 = (1 << 64) - 1


def _splitmix64_next(state: int):
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Rng:
    """xoshiro256** seeded through splitmix64."""

    __slots__ = ("s0", "s1", "s2", "s3")

    def __init__(self, seed: int):
        st = seed & MASK64
        st, self.s0 = _splitmix64_next(st)
        st, self.s1 = _splitmix64_next(st)
        st, self.s2 = _splitmix64_next(st)
        st, self.s3 = _splitmix64_next(st)

    def next_u64(self) -> int:
        s0, s1, s2, s3 = self.s0, self.s1, self.s2, self.s3
        result = (_rotl((s1 * 5) & MASK64, 7) * 9) & MASK64
        t = (s1 << 17) & MASK64
        s2 ^= s0
        s3 ^= s1
        s1 ^= s2
        s0 ^= s3
        s2 ^= t
        s3 = _rotl(s3, 45)
        self.s0, self.s1, self.s2, self.s3 = s0, s1, s2, s3
        return result

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, a: int, b: int) -> int:
        """Uniform integer on {a..b} (inclusive)."""
        return a + int(math.floor(self.uniform() * (b - a + 1)))


def _empty(n: int) -> List[int]:
    return [0] * n


def _add_edge(adj: List[int], i: int, j: int) -> None:
    adj[i] |= 1 << j
    adj[j] |= 1 << i


def gnp(n: int, p: float, seed: int, rng: Rng | None = None) -> List[int]:
    rng = rng or Rng(seed)
    adj = _empty(n)
    for i in range(n):
        for j in range(i + 1, n):
            if rng.uniform() < p:
                _add_edge(adj, i, j)
    return adj


def rgg(n: int, r: float, seed: int, rng: Rng | None = None) -> List[int]:
    rng = rng or Rng(seed)
    pts = []
    for _ in range(n):
        x = rng.uniform()
        y = rng.uniform()
        pts.append((x, y))
    r2 = r * r
    adj = _empty(n)
    for i in range(n):
        xi, yi = pts[i]
        for j in range(i + 1, n):
            dx = xi - pts[j][0]
            dy = yi - pts[j][1]
            if dx * dx + dy * dy <= r2:
                _add_edge(adj, i, j)
    return adj


def ktree(n: int, k: int, seed: int, rng: Rng | None = None) -> List[int]:
    """Random k-tree on n >= k+1 vertices."""
    if n < k + 1:
        raise ValueError("a k-tree needs n >= k+1")
    rng = rng or Rng(seed)
    adj = _empty(n)
    base = list(range(k + 1))
    for i in base:
        for j in base:
            if i < j:
                _add_edge(adj, i, j)
    cliques: List[List[int]] = [[u for u in base if u != drop] for drop in base]
    for v in range(k + 1, n):
        c = cliques[int(math.floor(rng.uniform() * len(cliques)))]
        for u in c:
            _add_edge(adj, u, v)
        for w in c:
            cliques.append(sorted([u for u in c if u != w] + [v]))
    return adj


def edges_of(adj: Sequence[int]) -> List[tuple]:
    n = len(adj)
    return [(i, j) for i in range(n) for j in range(i + 1, n) if (adj[i] >> j) & 1]


def partial_ktree(n: int, k: int, seed: int, remove_frac: float = 0.3,
                  rng: Rng | None = None) -> List[int]:
    rng = rng or Rng(seed)
    adj = ktree(n, k, seed, rng=rng)
    edges = edges_of(adj)
    m = len(edges)
    for idx in range(m - 1, 0, -1):
        j = int(math.floor(rng.uniform() * (idx + 1)))
        edges[idx], edges[j] = edges[j], edges[idx]
    n_remove = int(math.floor(remove_frac * m + 0.5))
    for (i, j) in edges[:n_remove]:
        adj[i] &= ~(1 << j)
        adj[j] &= ~(1 << i)
    return adj


# ---------------------------------------------------------------- families
def mixed_graph(seed: int, n_lo: int, n_hi: int, gnp_family: bool) -> List[int]:
    """One graph of the mixed G(n,p) / partial k-tree family.

    G(n,p): n ~ U{n_lo..n_hi}, p ~ U[0.1, 0.5].  Partial k-tree: k ~ U{3..12},
    n ~ U{max(n_lo, k+2)..n_hi}, 30% of the edges removed.  The parameters are
    drawn from the graph's own stream before the graph itself.
    """
    rng = Rng(seed)
    if gnp_family:
        n = rng.randint(n_lo, n_hi)
        p = 0.1 + 0.4 * rng.uniform()
        return gnp(n, p, seed, rng=rng)
    k = rng.randint(3, 12)
    n = rng.randint(max(n_lo, k + 2), n_hi)
    return partial_ktree(n, k, seed, rng=rng)


def batch_graphs(count: int = 4096, seed0: int = 0, n_lo: int = 16, n_hi: int = 48) -> List[List[int]]:
    """The batched workload: graph g (seed seed0+g) is G(n,p) when g is even,
    otherwise a partial k-tree."""
    return [mixed_graph(seed0 + g, n_lo, n_hi, g % 2 == 0) for g in range(count)]


def learned_k_train(count: int = 20000) -> List[List[int]]:
    """Training graphs of the learned-k workload: seeds 10^6 + j, n in [12, 40]."""
    return [mixed_graph(10**6 + j, 12, 40, j % 2 == 0) for j in range(count)]


def learned_k_test(count: int = 2000) -> List[List[int]]:
    """Held-out graphs of the learned-k workload: seeds 2*10^6 + j, n in [30, 56]."""
    return [mixed_graph(2 * 10**6 + j, 30, 56, j % 2 == 0) for j in range(count)]


# ------------------------------------------------------------ named inputs
def workload_gnp20() -> List[int]:
    """Single Erdos-Renyi graph G(n=20, p=0.3), seed 0."""
    return gnp(20, 0.3, 0)


def workload_rgg40() -> List[int]:
    """Single random geometric graph, n=40, radius 0.25, seed 0."""
    return rgg(40, 0.25, 0)


def workload_pktree60() -> List[int]:
    """Partial 10-tree, n=60, 30% of the edges removed, seed 0."""
    return partial_ktree(60, 10, 0)


# ------------------------------------------------------------- structured
def complete(n: int) -> List[int]:
    full = (1 << n) - 1
    return [full & ~(1 << i) for i in range(n)]


def path(n: int) -> List[int]:
    adj = _empty(n)
    for i in range(n - 1):
        _add_edge(adj, i, i + 1)
    return adj


def cycle(n: int) -> List[int]:
    adj = path(n)
    if n >= 3:
        _add_edge(adj, 0, n - 1)
    return adj


def star(n: int) -> List[int]:
    adj = _empty(n)
    for i in range(1, n):
        _add_edge(adj, 0, i)
    return adj


def grid(a: int, b: int) -> List[int]:
    adj = _empty(a * b)
    for r in range(a):
        for c in range(b):
            v = r * b + c
            if c + 1 < b:
                _add_edge(adj, v, v + 1)
            if r + 1 < a:
                _add_edge(adj, v, v + b)
    return adj


def complete_bipartite(a: int, b: int) -> List[int]:
    adj = _empty(a + b)
    for i in range(a):
        for j in range(a, a + b):
            _add_edge(adj, i, j)
    return adj


def random_tree(n: int, seed: int) -> List[int]:
    rng = Rng(seed)
    adj = _empty(n)
    for v in range(1, n):
        _add_edge(adj, v, rng.randint(0, v - 1))
    return adj


def relabel(adj: Sequence[int], seed: int) -> List[int]:
    """The same graph under a seeded random vertex permutation."""
    n = len(adj)
    rng = Rng(seed)
    perm = list(range(n))
    for idx in range(n - 1, 0, -1):
        j = int(math.floor(rng.uniform() * (idx + 1)))
        perm[idx], perm[j] = perm[j], perm[idx]
    out = _empty(n)
    for i in range(n):
        row = adj[i]
        while row:
            j = (row & -row).bit_length() - 1
            row &= row - 1
            out[perm[i]] |= 1 << perm[j]
    return out


# ---------------------------------------------------------------- layouts
def words_for(n: int) -> int:
    return max(1, (n + 63) // 64)


def to_rows_u64(adj: Sequence[int], words: int | None = None) -> np.ndarray:
    """n x ceil(n/64) little-endian uint64 words (bit c of row r = edge rc)."""
    n = len(adj)
    w = words or words_for(n)
    out = np.zeros((n, w), dtype=np.uint64)
    for i, row in enumerate(adj):
        for j in range(w):
            out[i, j] = (row >> (64 * j)) & MASK64
    return out


def to_rows_u32(adj: Sequence[int]) -> np.ndarray:
    n = len(adj)
    if n > 32:
        raise ValueError("uint32 rows hold at most 32 vertices")
    return np.array([row & 0xFFFFFFFF for row in adj], dtype=np.uint32)


def concat_rows_u64(graphs: Sequence[Sequence[int]]):
    """Concatenated uint64 rows of many graphs plus (n, row_offset) arrays.

    Graph g's rows start at word ``row_offset[g]``; each of its n[g] rows has
    ceil(n[g]/64) words."""
    ns = np.array([len(g) for g in graphs], dtype=np.int32)
    offs = np.zeros(len(graphs), dtype=np.int64)
    total = 0
    for g, adj in enumerate(graphs):
        offs[g] = total
        total += len(adj) * words_for(len(adj))
    out = np.zeros(total, dtype=np.uint64)
    for g, adj in enumerate(graphs):
        w = words_for(len(adj))
        out[offs[g]: offs[g] + len(adj) * w] = to_rows_u64(adj, w).reshape(-1)
    return out, ns, offs
