"""Shared helpers of the GPU tests (test code only)."""
import numpy as np
import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg


def context(**kw):
    from paper_1709_09990_gb300 import native
    return native.Context(device=0, **kw)


def assert_decide_matches(ctx, adj, k, check_order=True):
    exp = oracle.decide(adj, k, count_canonical=True)
    got = ctx.decide(adj, k=k, want_order=check_order)
    st = got["stats"]
    assert got["yes"] == exp["yes"], (k, got["yes"], exp["yes"])
    assert st["levels"] == exp["levels"], (k, st["level_size"], exp["level_size"])
    assert st["level_size"] == exp["level_size"], k
    assert st["fp_sum"] == exp["fp_sum"], k
    assert st["fp_xor"] == exp["fp_xor"], k
    assert st["states_expanded"] == exp["states_expanded"]
    assert st["candidates"] == exp["candidates"]
    # the GPU submits only the canonical pairs to its table
    assert st["generated"] == exp["canonical"]
    if check_order and got["yes"]:
        order = got["order"].tolist()
        assert sorted(order) == list(range(len(adj)))
        assert oracle.width_q(adj, order) <= k
        assert oracle.width_elim(adj, order) <= k
    return got, exp


def fingerprint_sums(keys: np.ndarray):
    """Sum (mod 2^64) and xor of the splitmix64 output function over 64-bit
    keys: the level digest the libtw counters and the oracle report."""
    z = keys.astype(np.uint64).reshape(-1)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
        s = int(np.sum(z, dtype=np.uint64))
    return s, int(np.bitwise_xor.reduce(z)) if z.size else 0
