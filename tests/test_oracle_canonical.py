"""Pins of the canonical-parent counter and of the fact behind it.

The CUDA path extends a set S by v only when v lies in the component of
G[S u {v}] that holds the lowest vertex of S u {v}.  That keeps every level
set unchanged because feasibility splits over components: Q(S, v) depends
only on the component of G[S u {v}] that contains v (Section 2's definition of
Q: the interior of each path lies in S), so a set is feasible iff each
component of it is, and the last vertex of a feasible ordering of the
lowest-vertex component is a parent of that kind.

These tests check the fact itself by brute force in plain Python (whole level
sets, tiny graphs), and the oracle's ``canonical`` counter against the same
brute force and against a closed form.
"""
import math

import oracle
from paper_1709_09990_gb300 import graphgen as gg


def _q(adj, s, v):
    """Q(S, v) by a search from v through S (Section 2)."""
    seen, stack, q = {v}, [v], set()
    while stack:
        u = stack.pop()
        for w in range(len(adj)):
            if (adj[u] >> w) & 1 and w not in seen:
                seen.add(w)
                if (s >> w) & 1:
                    stack.append(w)
                else:
                    q.add(w)
    return q


def _holds_lowest(adj, s, v):
    t = s | (1 << v)
    low = (t & -t).bit_length() - 1
    seen, stack = {v}, [v]
    while stack:
        u = stack.pop()
        for w in range(len(adj)):
            if (adj[u] >> w) & 1 and (t >> w) & 1 and w not in seen:
                seen.add(w)
                stack.append(w)
    return low in seen


def _levels(adj, k, canonical_only):
    """Listing 1 with whole sets; optionally only canonical extensions."""
    n = len(adj)
    level, out, pairs = {0}, [{0}], 0
    for _ in range(n - k - 1):
        nxt = set()
        for s in level:
            for v in range(n):
                if (s >> v) & 1 or len(_q(adj, s, v)) > k:
                    continue
                if canonical_only and not _holds_lowest(adj, s, v):
                    continue
                pairs += 1
                nxt.add(s | (1 << v))
        level = nxt
        out.append(level)
        if not level:
            break
    return out, pairs


def _small_graphs():
    graphs = []
    for s in range(60):
        rng = gg.Rng(900 + s)
        n = rng.randint(1, 8)
        graphs.append(gg.gnp(n, 0.15 + 0.7 * rng.uniform(), 900 + s, rng=rng))
    graphs += [gg.path(7), gg.cycle(7), gg.star(7), [0] * 6, gg.partial_ktree(8, 3, 2)]
    return graphs


def test_canonical_extensions_give_the_same_level_sets():
    for adj in _small_graphs():
        for k in range(len(adj)):
            full, _ = _levels(adj, k, False)
            canon, _ = _levels(adj, k, True)
            assert canon == full, (adj, k)


def test_oracle_counters_match_brute_force():
    for adj in _small_graphs():
        for k in range(len(adj)):
            full, f_pairs = _levels(adj, k, False)
            _, c_pairs = _levels(adj, k, True)
            d = oracle.decide(adj, k, count_canonical=True)
            assert d["level_size"] == [len(x) for x in full], (adj, k)
            assert d["feasible"] == f_pairs, (adj, k)
            assert d["canonical"] == c_pairs, (adj, k)


def test_edgeless_closed_form():
    # Every set is feasible at k = 0 and its components are single vertices,
    # so each set T of levels 1 .. n-1 has exactly one canonical parent,
    # T minus its lowest vertex: 2^n - 2 pairs; all n-i extensions of the
    # C(n, i) sets of level i are feasible.
    for n in (3, 6, 11):
        d = oracle.decide([0] * n, 0, count_canonical=True)
        assert d["canonical"] == 2 ** n - 2
        assert d["feasible"] == sum(math.comb(n, i) * (n - i) for i in range(n - 1))


def test_canonical_count_bounds():
    # between one pair per non-empty set of the later levels and all
    # feasible pairs
    for adj in (gg.workload_gnp20(), gg.gnp(14, 0.4, 7), gg.partial_ktree(16, 4, 1)):
        for k in (3, 5, 7):
            d = oracle.decide(adj, k, count_canonical=True)
            assert sum(d["level_size"][1:]) <= d["canonical"] <= d["feasible"]
            plain = oracle.decide(adj, k)
            assert plain["level_size"] == d["level_size"] and plain["feasible"] == d["feasible"]


def test_oracle_level_keys_are_the_brute_force_sets():
    # the sets the oracle exports for element-wise GPU checks are the whole
    # level sets of the plain-Python brute force, level by level
    for adj in _small_graphs()[::3]:
        n = len(adj)
        for k in range(n):
            full, _ = _levels(adj, k, False)
            for i, lvl in enumerate(full):
                keys = oracle.level_keys(adj, k, i)
                assert [int(r[0]) for r in keys] == sorted(lvl), (adj, k, i)
            assert len(oracle.level_keys(adj, k, len(full))) == 0
    # two words per set beyond 64 vertices: the star K_{1,69} at k = 1
    star = gg.star(70)
    keys = oracle.level_keys(star, 1, 2)
    assert keys.shape == (math.comb(69, 2), 2)
    got = {int(r[0]) | (int(r[1]) << 64) for r in keys}
    assert got == {(1 << a) | (1 << b) for a in range(1, 70) for b in range(a + 1, 70)}
