"""GPU solve (k sweep, ordering, tree decomposition), bounds, capacity and
robustness paths, device-pointer inputs."""
import numpy as np
import pytest

import oracle
from oracle import bounds as obounds
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def _check_solution(adj, sol, tw):
    assert sol["tw"] == tw
    order = sol["order"].tolist()
    assert oracle.width_q(adj, order) == tw
    assert oracle.verify_td(adj, sol["td_parent"], sol["td_bags"]) == tw


@pytest.mark.parametrize("seed", range(4))
def test_solve_random(ctx, seed):
    rng = gg.Rng(700 + seed)
    for _ in range(6):
        n = rng.randint(1, 30)
        adj = gg.gnp(n, 0.1 + 0.5 * rng.uniform(), rng.next_u64())
        ref = oracle.solve(adj, want_order=False)
        sol = ctx.solve(adj, want_order=True, want_td=True)
        _check_solution(adj, sol, ref["tw"])


def test_solve_families(ctx):
    cases = [gg.grid(4, 5), gg.complete_bipartite(4, 6), gg.cycle(20), gg.random_tree(20, 3), gg.complete(12),
             gg.ktree(26, 4, 2), gg.partial_ktree(26, 5, 3), [0] * 7]
    closed = [4, 4, 2, 1, 11, 4, None, 0]
    for adj, tw in zip(cases, closed):
        sol = ctx.solve(adj, want_order=True, want_td=True)
        if tw is None:
            tw = oracle.solve(adj, want_order=False)["tw"]
        _check_solution(adj, sol, tw)


def test_solve_gnp20_sweep_counters(ctx):
    adj = gg.workload_gnp20()
    lb = max(obounds.mmd(adj), obounds.mmd_plus(adj))
    ref = oracle.solve(adj, k_start=lb, want_order=False)
    sol = ctx.solve(adj, want_order=True, want_td=True)
    _check_solution(adj, sol, ref["tw"])
    assert sol["stats"]["states_expanded"] == ref["states_expanded"]
    assert sol["stats"]["decide_runs"] == ref["k_tried"]


@pytest.mark.parametrize("seed", range(3))
def test_bounds_match_oracle(ctx, seed):
    rng = gg.Rng(900 + seed)
    for _ in range(10):
        n = rng.randint(2, 100)
        adj = gg.gnp(n, 0.05 + 0.5 * rng.uniform(), rng.next_u64())
        got = ctx.bounds(adj).tolist()
        exp = [obounds.mmd(adj), obounds.mmd_plus(adj), obounds.min_degree_ub(adj), obounds.min_fill_ub(adj)]
        assert got == exp, (n, got, exp)


def test_features_match_oracle(ctx):
    graphs = [gg.mixed_graph(5000 + j, 12, 56, j % 2 == 0) for j in range(40)] + [gg.complete(9), gg.star(11)]
    got = ctx.features(graphs)
    exp = np.array([obounds.features(a) for a in graphs], dtype=np.float64)
    np.testing.assert_allclose(got, exp.astype(np.float32), rtol=1e-6, atol=1e-7)


def test_capacity_error_is_reported_not_wrong():
    from paper_1709_09990_gb300 import native
    adj = gg.workload_rgg40()
    with context(mem_cap_bytes=1 << 20) as small:
        with pytest.raises(native.TwError) as e:
            small.decide(adj, k=6)
        assert e.value.status == native.TW_ERR_CAPACITY
        # the context stays usable after the error
        got = small.decide(gg.workload_gnp20(), k=8)
        assert got["yes"]


def test_tiny_probe_limit_and_load_still_exact():
    adj = gg.workload_gnp20()
    exp = oracle.decide(adj, 8)
    with context(max_probes=2, table_load_pct=90, fingerprints=True) as c:
        got = c.decide(adj, k=8)
        assert got["stats"]["level_size"] == exp["level_size"]
        assert got["stats"]["fp_sum"] == exp["fp_sum"]


@pytest.mark.parametrize("bt", [64, 128, 256])
def test_block_sizes(bt):
    adj = gg.workload_gnp20()
    exp = oracle.decide(adj, 8)
    with context(block_threads=bt, fingerprints=True) as c:
        got = c.decide(adj, k=8)
        assert got["stats"]["level_size"] == exp["level_size"]
        assert got["stats"]["fp_xor"] == exp["fp_xor"]


def test_device_pointer_inputs_and_outputs(ctx):
    torch = pytest.importorskip("torch")
    adj = gg.workload_gnp20()
    rows = torch.from_numpy(gg.to_rows_u64(adj).astype(np.int64)).cuda()
    tw_d = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    order_d = torch.full((20,), -1, dtype=torch.int32, device="cuda")
    sol = ctx.solve(rows, n=20, tw_out=tw_d, order_out=order_d)
    torch.cuda.synchronize()
    ref = oracle.solve(adj, want_order=False)["tw"]
    assert int(tw_d.item()) == ref
    assert oracle.width_q(adj, order_d.cpu().tolist()) == ref


def test_batch_loop_matches_oracle(ctx):
    graphs = [gg.mixed_graph(77 + j, 10, 22, j % 2 == 0) for j in range(24)]
    res = ctx.solve_batch(graphs)
    assert res["status"] == 0
    pos = 0
    for g, adj in enumerate(graphs):
        tw = oracle.solve(adj, want_order=False)["tw"]
        assert res["tw"][g] == tw
        order = res["orders"][pos: pos + len(adj)].tolist()
        assert oracle.width_q(adj, order) == tw
        pos += len(adj)


def test_batch_with_hints_is_exact(ctx):
    graphs = [gg.mixed_graph(300 + j, 10, 22, j % 2 == 0) for j in range(16)]
    exact = [oracle.solve(a, want_order=False)["tw"] for a in graphs]
    for shift in (-3, 0, 2):
        hint = np.array([t + shift for t in exact], dtype=np.float32)
        res = ctx.solve_batch(graphs, k_hint=hint)
        assert res["status"] == 0
        assert res["tw"].tolist() == exact


def test_batched_path_mixed_sizes_and_hints(ctx):
    # graphs of 10..64 vertices go through the batched kernel, larger ones
    # through the single-graph path; tw must equal the oracle's for all
    graphs = [gg.mixed_graph(900 + j, 10, 26, j % 2 == 0) for j in range(60)]
    graphs += [gg.gnp(60, 0.7, 12), gg.gnp(70, 0.8, 110), gg.complete(5), [0], gg.path(33)]
    exact = []
    for a in graphs:
        lb = max(obounds.mmd(a), obounds.mmd_plus(a))
        exact.append(oracle.solve(a, k_start=lb, want_order=False)["tw"])
    for hint in (None, np.array(exact, np.float32) + 2, np.array(exact, np.float32) - 2):
        res = ctx.solve_batch(graphs, k_hint=hint)
        assert res["status"] == 0
        assert res["tw"].tolist() == exact
        pos = 0
        for g, adj in enumerate(graphs):
            order = res["orders"][pos: pos + len(adj)].tolist()
            assert oracle.width_q(adj, order) == exact[g]
            pos += len(adj)


def test_batched_path_evicts_large_levels(ctx):
    # the geometric n=40 graph has levels of ~5.9 M states: it leaves the
    # batch and is finished by the single-graph path
    graphs = [gg.workload_gnp20(), gg.workload_rgg40(), gg.cycle(12)]
    res = ctx.solve_batch(graphs)
    assert res["status"] == 0
    assert res["tw"].tolist() == [8, 6, 2]
    assert res["stats"]["states_expanded"] >= 79399414


def test_autotuned_run_is_exact():
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rgg40_seed0_k6.json")))["decide"][0]
    adj = gg.workload_rgg40()
    with context(autotune=True, fingerprints=True) as c:
        for _ in range(2):  # the first run tunes on its first level of >= 2^18 states
            got = c.decide(adj, k=6)
            assert got["stats"]["level_size"] == rec["level_size"]
            assert [str(x) for x in got["stats"]["fp_xor"]] == rec["fp_xor"]
