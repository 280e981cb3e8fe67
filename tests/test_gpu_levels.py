"""Element-by-element parity of whole wavefront levels (Section 3.1).

The other parity tests compare each level through its size and a set
fingerprint.  Here the GPU's level is downloaded through tw_decide_level and
its sets, sorted, must equal the oracle's sorted sets exactly, for each state
width: 32-bit (G(20, 0.3)), 64-bit (the n = 40 geometric benchmark graph at
k = 6, levels of 190,183 and 391,643 states) and 128-bit (a partial 3-tree
with n = 70, a level of 216,489 states).
"""
import numpy as np
import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


def _gpu_level(ctx, adj, k, level):
    r = ctx.decide_level(adj, k=k, level=level)
    return oracle.sort_keys(r["keys"]), r


@pytest.mark.parametrize("case", [("gnp20", 8, 6), ("gnp20", 7, 9), ("rgg40", 6, 7), ("rgg40", 6, 8),
                                  ("pktree70", 3, 4)])
def test_level_sets_equal_oracle_element_by_element(case):
    name, k, level = case
    adj = {"gnp20": gg.workload_gnp20, "rgg40": gg.workload_rgg40,
           "pktree70": lambda: gg.partial_ktree(70, 3, 5)}[name]()
    exp = oracle.level_keys(adj, k, level)
    with context() as ctx:
        got, r = _gpu_level(ctx, adj, k, level)
    assert r["count"] == len(exp)
    assert got.shape == exp.shape
    assert np.array_equal(got, exp)
    # every set has exactly `level` vertices and no vertex >= n
    n = len(adj)
    pop = sum(np.array([bin(int(x)).count("1") for x in got[:, j]]) for j in range(got.shape[1]))
    assert np.all(pop == level)
    if n < 64:
        assert np.all(got[:, 0] >> np.uint64(n) == 0)


def test_level_edges():
    adj = gg.workload_gnp20()
    with context() as ctx:
        # level 0 is the empty set
        got, r = _gpu_level(ctx, adj, 8, 0)
        assert r["count"] == 1 and got.tolist() == [[0]]
        # K_6 at k = 3: level 1 is already empty, later levels do not exist
        k6 = gg.complete(6)
        assert ctx.decide_level(k6, k=3, level=1)["count"] == 0
        assert ctx.decide_level(k6, k=3, level=2)["count"] == 0
        # a buffer smaller than the level: capacity status, true count
        from paper_1709_09990_gb300 import native
        small = np.zeros((3, 1), np.uint64)
        with pytest.raises(native.TwError) as e:
            ctx.decide_level(adj, k=8, level=2, keys_out=small)
        assert e.value.status == native.TW_ERR_CAPACITY
        # into a device tensor
        torch = pytest.importorskip("torch")
        exp = oracle.level_keys(adj, 8, 3)
        dev = torch.zeros((len(exp), 1), dtype=torch.int64, device="cuda:0")
        r = ctx.decide_level(adj, k=8, level=3, keys_out=dev)
        got = oracle.sort_keys(r["keys"].cpu().numpy().view(np.uint64))
        assert np.array_equal(got, exp)
