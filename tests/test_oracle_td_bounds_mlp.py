"""Pins of the oracle's tree-decomposition checker, bounds and network."""
import numpy as np
import pytest

import oracle
from oracle import bounds, mlp
from paper_1709_09990_gb300 import graphgen as gg


def test_td_from_optimal_order_verifies():
    for s in range(30):
        adj = gg.gnp(12, 0.3, 2000 + s)
        res = oracle.solve(adj)
        width, parent, bags = oracle.td_from_order(adj, res["order"])
        assert width == res["tw"]
        assert oracle.verify_td(adj, parent, bags) == res["tw"]


def test_td_checker_rejects_planted_mistakes():
    adj = gg.grid(3, 4)
    res = oracle.solve(adj)
    width, parent, bags = oracle.td_from_order(adj, res["order"])
    assert oracle.verify_td(adj, parent, bags) == 3
    # an edge no bag covers
    for v in range(12):
        b = bags.copy()
        nb = adj[v]
        if nb:
            u = (nb & -nb).bit_length() - 1
            # drop u from every bag that holds v
            for x in range(12):
                if (int(b[x, 0]) >> v) & 1 and x != u:
                    b[x, 0] = np.uint64(int(b[x, 0]) & ~(1 << u))
            if oracle.verify_td(adj, parent, b) == -1:
                break
    else:
        pytest.fail("checker accepted a decomposition without edge cover")
    # two roots
    idx = int(np.nonzero(parent != -1)[0][0])
    p = parent.copy(); p[idx] = -1
    assert oracle.verify_td(adj, p, bags) == -1
    # a cycle in the parent pointers
    p = parent.copy(); root = int(np.nonzero(parent == -1)[0][0]); p[root] = idx
    assert oracle.verify_td(adj, p, bags) == -1
    # a vertex in no bag
    b = bags.copy(); b[:, 0] &= np.uint64(~1 & 0xFFFFFFFFFFFFFFFF)
    assert oracle.verify_td(adj, parent, b) == -1


def test_td_running_intersection_violation():
    # path 0-1-2 ; bags {0,1} -> {2} -> {1,2}: vertex 1 appears in two bags
    # separated by a bag without it.
    adj = gg.path(3)
    bags = np.array([[0b011], [0b100], [0b110]], dtype=np.uint64)
    parent = np.array([1, 2, -1], dtype=np.int32)
    assert oracle.verify_td(adj, parent, bags) == -1
    bags_ok = np.array([[0b011], [0b110], [0b100]], dtype=np.uint64)
    assert oracle.verify_td(adj, parent, bags_ok) == 1


def test_bounds_closed_forms():
    for n in range(2, 9):
        k = gg.complete(n)
        assert bounds.mmd(k) == bounds.mmd_plus(k) == bounds.min_degree_ub(k) == bounds.min_fill_ub(k) == n - 1
    assert bounds.mmd(gg.path(6)) == 1 and bounds.min_fill_ub(gg.path(6)) == 1
    assert bounds.mmd(gg.cycle(7)) == 2 and bounds.mmd_plus(gg.cycle(7)) == 2
    # a grid's degeneracy is 2, but contractions reach larger minimum degree
    g = gg.grid(4, 4)
    assert bounds.mmd(g) == 2 and bounds.mmd_plus(g) >= 3
    assert bounds.min_fill_ub([0, 0, 0]) == 0


def test_bounds_sandwich_treewidth():
    for s in range(40):
        adj = gg.gnp(11, 0.2 + 0.5 * gg.Rng(s).uniform(), 3000 + s)
        tw = oracle.solve(adj, want_order=False)["tw"]
        assert bounds.mmd(adj) <= bounds.mmd_plus(adj) <= tw
        assert tw <= bounds.min_degree_ub(adj) and tw <= bounds.min_fill_ub(adj)


def test_features_closed_form():
    f = bounds.features(gg.complete(8))
    assert f[0] == 8 / 64 and f[1] == 1.0
    assert f[2] == f[3] == f[4] == 7 / 8 and f[5] == 0.0
    assert f[6:10] == [0.0, 0.0, 0.0, 1.0]
    assert f[10] == 7 / 8 and f[11] == 7 / 8
    f = bounds.features(gg.star(8))
    assert f[6:10] == [7 / 8, 0.0, 0.0, 1 / 8]


def _params(seed):
    rng = gg.Rng(seed)
    return np.array([rng.uniform() - 0.5 for _ in range(mlp.N_PARAMS)])


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.random((17, 12))
    y = rng.random(17)
    p = _params(1)
    g = mlp.grad(p, X, y)
    eps = 1e-6
    for idx in list(range(0, mlp.N_PARAMS, 7)) + [mlp.N_PARAMS - 1]:
        e = np.zeros(mlp.N_PARAMS); e[idx] = eps
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_mlp_forward_matches_loops():
    rng = np.random.default_rng(1)
    X = rng.random((5, 12))
    p = _params(2)
    W1, b1, W2, b2 = mlp.unpack(p)
    _, _, yhat = mlp.forward(p, X)
    for b in range(5):
        h = [max(0.0, sum(W1[j, i] * X[b, i] for i in range(12)) + b1[j]) for j in range(32)]
        assert abs(sum(W2[j] * h[j] for j in range(32)) + b2 - yhat[b]) < 1e-12


def test_adam_first_step_is_sign_step():
    # after one step from m = v = 0, bias correction gives p -= lr * g/(|g|+eps)
    p = np.zeros(4); g = np.array([1.0, -2.0, 0.5, 0.0])
    p2, m, v = mlp.adam_step(p, g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    assert np.allclose(p2, [-0.1, 0.1, -0.1, 0.0], atol=1e-6)
