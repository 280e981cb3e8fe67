"""The seeded input generators (input generation only, shared by the oracle
and the CUDA path): the published first splitmix64 output, the xoshiro256**
draws' range and moments, and structural facts of every family."""
import math

import oracle
from paper_1709_09990_gb300 import graphgen as gg


def _simple(adj):
    n = len(adj)
    for i in range(n):
        assert not (adj[i] >> i) & 1
        assert adj[i] >> n == 0
        for j in range(n):
            assert ((adj[i] >> j) & 1) == ((adj[j] >> i) & 1)


def test_splitmix64_first_output():
    # the first output of splitmix64 from seed 0 (Steele, Lea & Flood 2014)
    _, z = gg._splitmix64_next(0)
    assert z == 0xE220A8397B1DCDAF


def test_uniform_draws():
    rng = gg.Rng(12345)
    u = [rng.uniform() for _ in range(200000)]
    assert min(u) >= 0.0 and max(u) < 1.0
    mean = sum(u) / len(u)
    var = sum((x - mean) ** 2 for x in u) / len(u)
    assert abs(mean - 0.5) < 0.005          # sd of the mean: 0.00065
    assert abs(var - 1.0 / 12.0) < 0.002
    r = gg.Rng(7)
    ints = [r.randint(3, 12) for _ in range(20000)]
    assert min(ints) == 3 and max(ints) == 12
    # same seed, same stream; another seed, another stream
    assert [gg.Rng(5).next_u64() for _ in range(3)] == [gg.Rng(5).next_u64() for _ in range(3)]
    a, b = gg.Rng(5), gg.Rng(6)
    assert [a.next_u64() for _ in range(3)] != [b.next_u64() for _ in range(3)]


def test_gnp_density():
    adj = gg.gnp(200, 0.3, 4)
    _simple(adj)
    m = len(gg.edges_of(adj))
    pairs = 200 * 199 // 2
    assert abs(m - 0.3 * pairs) < 4 * math.sqrt(pairs * 0.3 * 0.7)
    assert gg.gnp(30, 0.0, 1) == [0] * 30
    assert gg.gnp(30, 1.0, 1) == gg.complete(30)


def test_geometric_graph_is_monotone_in_the_radius():
    small, large = gg.rgg(60, 0.15, 9), gg.rgg(60, 0.3, 9)  # same points
    _simple(large)
    for i in range(60):
        assert small[i] & ~large[i] == 0
    assert gg.rgg(25, 1.5, 3) == gg.complete(25)  # every distance is <= sqrt(2)


def test_ktree_structure():
    for n, k, seed in ((10, 3, 1), (14, 2, 5), (9, 4, 2), (30, 6, 8)):
        adj = gg.ktree(n, k, seed)
        _simple(adj)
        assert len(gg.edges_of(adj)) == k * (k + 1) // 2 + (n - k - 1) * k
        if n <= 10:
            assert oracle.brute_force_tw(adj) == k
        else:
            assert oracle.solve(adj, want_order=False)["tw"] == k


def test_partial_ktree_removes_a_fraction_of_the_ktree_edges():
    for n, k, seed in ((20, 4, 3), (60, 10, 0)):
        full = gg.ktree(n, k, seed)
        part = gg.partial_ktree(n, k, seed)
        _simple(part)
        m = len(gg.edges_of(full))
        assert len(gg.edges_of(part)) == m - int(math.floor(0.3 * m + 0.5))
        for i in range(n):
            assert part[i] & ~full[i] == 0


def test_workload_families():
    graphs = gg.batch_graphs(64)
    assert graphs == gg.batch_graphs(64)
    for g, adj in enumerate(graphs):
        _simple(adj)
        assert 16 <= len(adj) <= 48
    assert all(12 <= len(a) <= 40 for a in gg.learned_k_train(50))
    assert all(30 <= len(a) <= 56 for a in gg.learned_k_test(50))
    assert len(gg.workload_gnp20()) == 20 and len(gg.workload_rgg40()) == 40
    assert len(gg.workload_pktree60()) == 60
