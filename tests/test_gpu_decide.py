"""GPU decide(k) against the CPU oracle: answers, per-level sizes, level
fingerprints, counters and orderings, for all three state widths."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import bounds as obounds
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import assert_decide_matches, context

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = context(fingerprints=True)
    yield c
    c.close()


def test_gnp20_every_k(ctx):
    adj = gg.workload_gnp20()
    rec = json.load(open(os.path.join(GOLDEN, "gnp20_seed0.json")))
    for r in rec["decide"]:
        got = ctx.decide(adj, k=r["k"], want_order=True)
        st = got["stats"]
        assert got["yes"] == r["yes"]
        assert st["level_size"] == r["level_size"]
        assert [str(x) for x in st["fp_sum"]] == r["fp_sum"]
        assert [str(x) for x in st["fp_xor"]] == r["fp_xor"]
        assert st["states_expanded"] == r["states_expanded"]
        if got["yes"]:
            assert oracle.width_q(adj, got["order"].tolist()) <= r["k"]


def test_gnp20_u32_entry_point(ctx):
    adj = gg.workload_gnp20()
    rows = gg.to_rows_u32(adj)
    for k in (7, 8):
        exp = oracle.decide(adj, k)
        got = ctx.decide_u32(rows, 20, k, want_order=True)
        assert got["yes"] == exp["yes"]
        assert got["stats"]["level_size"] == exp["level_size"]
        assert got["stats"]["fp_sum"] == exp["fp_sum"]


@pytest.mark.parametrize("seed", range(6))
def test_random_small_u32(ctx, seed):
    rng = gg.Rng(100 + seed)
    for _ in range(8):
        n = rng.randint(2, 24)
        adj = gg.gnp(n, 0.1 + 0.6 * rng.uniform(), rng.next_u64(), rng=None)
        tw = oracle.solve(adj, want_order=False)["tw"]
        for k in sorted({max(0, tw - 2), max(0, tw - 1), tw, tw + 1}):
            assert_decide_matches(ctx, adj, k)


# 33 <= n <= 64, chosen so that each oracle run takes seconds
U64_CASES = [("gnp", 44, 0.5, 4), ("partial_ktree", 34, 8, 8), ("gnp", 50, 0.6, 11), ("gnp", 60, 0.7, 12),
             ("gnp", 64, 0.75, 14)]


@pytest.mark.parametrize("case", U64_CASES, ids=lambda c: f"{c[0]}{c[1]}")
def test_u64_class(ctx, case):
    fam, n, par, seed = case
    adj = getattr(gg, fam)(n, par, seed)
    lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
    tw = oracle.solve(adj, k_start=lb, want_order=False)["tw"]
    for k in (tw - 1, tw):
        assert_decide_matches(ctx, adj, k)


@pytest.mark.parametrize("case", [(66, 0.85), (70, 0.8), (80, 0.9), (90, 0.88), (100, 0.93), (128, 0.96)],
                         ids=lambda c: f"n{c[0]}")
def test_u128_class(ctx, case):
    # 65 <= n <= 128, dense enough that few levels are needed
    n, p = case
    adj = gg.gnp(n, p, 40 + n)
    lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
    tw = oracle.solve(adj, k_start=lb, want_order=False)["tw"]
    for k in (tw - 1, tw):
        assert_decide_matches(ctx, adj, k)


def test_u128_sparse_across_word_boundary(ctx):
    # a path on 70 vertices relabelled so that neighbours straddle bit 64
    adj = gg.relabel(gg.path(70), 5)
    for k in (0, 1):
        assert_decide_matches(ctx, adj, k)


def test_rgg40_small_k_golden(ctx):
    adj = gg.workload_rgg40()
    rec = json.load(open(os.path.join(GOLDEN, "rgg40_seed0_k4_k5.json")))
    for r in rec["decide"]:
        got = ctx.decide(adj, k=r["k"])
        assert got["yes"] == r["yes"]
        assert got["stats"]["level_size"] == r["level_size"]
        assert [str(x) for x in got["stats"]["fp_sum"]] == r["fp_sum"]
        assert got["stats"]["generated"] == r["canonical"]


def test_rgg40_full_k6_golden(ctx):
    path = os.path.join(GOLDEN, "rgg40_seed0_k6.json")
    if not os.path.exists(path):
        pytest.skip("k=6 record not generated")
    adj = gg.workload_rgg40()
    r = json.load(open(path))["decide"][0]
    got = ctx.decide(adj, k=6, want_order=True)
    assert got["yes"] == r["yes"]
    assert got["stats"]["level_size"] == r["level_size"]
    assert [str(x) for x in got["stats"]["fp_sum"]] == r["fp_sum"]
    assert [str(x) for x in got["stats"]["fp_xor"]] == r["fp_xor"]
    assert got["stats"]["states_expanded"] == r["states_expanded"]
    assert got["stats"]["generated"] == r["canonical"]
    assert oracle.width_q(adj, got["order"].tolist()) <= 6


def test_closed_form_levels(ctx):
    import math
    for n in (5, 17, 22):
        got = ctx.decide([0] * n, k=0)
        assert got["stats"]["level_size"] == [math.comb(n, i) for i in range(n)]
        got = ctx.decide(gg.cycle(n), k=2)
        assert got["stats"]["level_size"] == [math.comb(n, i) for i in range(n - 2)]
        got = ctx.decide(gg.star(n), k=1)
        assert got["stats"]["level_size"] == [math.comb(n - 1, i) for i in range(n - 1)]
    for n in (5, 17, 33, 40, 64, 65, 100, 128):
        got = ctx.decide(gg.path(n), k=1, want_order=True)
        assert got["stats"]["level_size"] == [i + 1 for i in range(n - 1)]
        assert oracle.width_q(gg.path(n), got["order"].tolist()) == 1
        got = ctx.decide(gg.complete(n), k=n - 2)
        assert got["stats"]["level_size"] == [1, 0] and not got["yes"]


def test_degenerate_inputs(ctx):
    got = ctx.decide([0], k=0, want_order=True)
    assert got["yes"] and got["order"].tolist() == [0] and got["stats"]["levels"] == 1
    adj = gg.gnp(9, 0.5, 1)
    got = ctx.decide(adj, k=8, want_order=True)  # k >= n-1
    assert got["yes"] and sorted(got["order"].tolist()) == list(range(9))
    from paper_1709_09990_gb300 import native
    bad = gg.to_rows_u64(adj)
    bad[0, 0] |= np.uint64(1 << 5) if not (int(bad[5, 0]) & 1) else np.uint64(0)
    bad[0, 0] ^= np.uint64(1 << 3)  # break symmetry
    with pytest.raises(native.TwError) as e:
        ctx.decide(bad, n=9, k=3)
    assert e.value.status == native.TW_ERR_INVALID
    loop = gg.to_rows_u64(adj)
    loop[2, 0] |= np.uint64(1 << 2)
    with pytest.raises(native.TwError):
        ctx.decide(loop, n=9, k=3)
    with pytest.raises(native.TwError):
        ctx.decide(adj, k=-1)


@pytest.mark.parametrize("case", ["gnp20", "u64", "u128", "rgg40_k5"])
def test_graph_driven_levels_match_host_loop(case):
    graphs = {"gnp20": (gg.workload_gnp20(), (6, 7, 8)), "u64": (gg.gnp(50, 0.6, 11), None),
              "u128": (gg.gnp(80, 0.9, 120), None), "rgg40_k5": (gg.workload_rgg40(), (4, 5))}
    adj, ks = graphs[case]
    if ks is None:
        lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
        tw = oracle.solve(adj, k_start=lb, want_order=False)["tw"]
        ks = (tw - 1, tw)
    with context(fingerprints=True, graph_levels=-1) as host, context(fingerprints=True, graph_levels=1) as graph:
        for k in ks:
            a = host.decide(adj, k=k, want_order=True)
            graph.decide(adj, k=k, want_order=True)  # first call grows the buffers
            b = graph.decide(adj, k=k, want_order=True)
            for key in ("level_size", "fp_sum", "fp_xor", "states_expanded", "candidates", "generated", "levels"):
                assert a["stats"][key] == b["stats"][key], (k, key)
            assert a["yes"] == b["yes"]
            if b["yes"]:
                assert oracle.width_q(adj, b["order"].tolist()) <= k


def test_graph_driven_solve_reuses_its_graphs():
    adj = gg.workload_gnp20()
    with context(graph_levels=1) as c:
        first = c.solve(adj, want_td=True)
        again = [c.solve(adj, want_td=True) for _ in range(3)]
    for r in again:
        assert r["tw"] == first["tw"] == 8
        assert r["stats"]["states_expanded"] == first["stats"]["states_expanded"]
        assert oracle.verify_td(adj, r["td_parent"], r["td_bags"]) == 8


def test_timed_graph_levels_report_expand_time():
    # time_kernels inside the graph-driven loop (event-record nodes around
    # every expand) and in the host loop: same levels, both timed
    adj = gg.workload_rgg40()
    with context(time_kernels=True, graph_levels=1, fingerprints=True) as a, \
            context(time_kernels=True, graph_levels=-1, fingerprints=True) as b:
        a.decide(adj, k=5)  # the first call grows the buffers
        ra, rb = a.decide(adj, k=5)["stats"], b.decide(adj, k=5)["stats"]
    for key in ("level_size", "fp_sum", "fp_xor", "generated", "expand_launches"):
        assert ra[key] == rb[key], key
    assert ra["expand_seconds"] > 0 and rb["expand_seconds"] > 0
