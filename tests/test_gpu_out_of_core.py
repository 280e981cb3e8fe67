"""Decide runs whose levels and tables exceed the memory cap (out_of_core).

With out_of_core, a level's hash table is built in slices, one hash range
per pass, and levels that do not fit the device go to pinned host memory
(Section 4.2's list capacity; the Conclusions' future work).  The runs below
use caps far below what the in-memory run needs and must give the same level
sets: the full decide(6) of the n = 40 benchmark graph (golden record,
79,399,414 states) under a 48 MB cap, and the first eleven levels of the
partial 10-tree n = 60 at k = 10 (level 10: 566,907,942 states, 4.5 GB of
keys) under a 1 GB cap.  With a host limit as well (host_cap_mb), the peak
levels of the n = 40 graph fit neither memory alone and are split between
device and host memory.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1709_09990_gb300 import graphgen as gg
from tests.gpu_util import context, fingerprint_sums

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_benchmark_run_under_a_48mb_cap_matches_the_golden_record():
    rec = json.load(open(os.path.join(GOLDEN, "rgg40_seed0_k6.json")))["decide"][0]
    adj = gg.workload_rgg40()
    with context(fingerprints=True, mem_cap_bytes=48 << 20, out_of_core=True) as ctx:
        r = ctx.decide(adj, k=6)
        st = r["stats"]
        assert r["yes"]
        assert st["level_size"] == rec["level_size"]
        assert st["fp_sum"] == [int(x) for x in rec["fp_sum"]]
        assert st["fp_xor"] == [int(x) for x in rec["fp_xor"]]
        assert st["states_expanded"] == rec["states_expanded"]
        assert st["generated"] == rec["canonical"]
        # some levels ran in several hash-range passes
        assert st["expand_launches"] > len(rec["level_size"]) - 1
    # without out_of_core the same cap is a capacity error
    with context(mem_cap_bytes=48 << 20) as ctx:
        assert ctx.decide(adj, k=6, raise_on_error=False)["status"] == 2


def test_partial_10tree_levels_under_a_1gb_cap():
    adj = gg.workload_pktree60()
    with context(fingerprints=True) as ctx:
        ref = ctx.decide(adj, k=10, raise_on_error=False)["stats"]  # in HBM up to the default cap
    assert len(ref["level_size"]) >= 11
    with context(fingerprints=True, mem_cap_bytes=1 << 30, out_of_core=True) as ctx:
        r = ctx.decide_level(adj, k=10, level=10, count_only=True)
    st = r["stats"]
    assert r["count"] == ref["level_size"][10] == 566_907_942
    assert st["level_size"] == ref["level_size"][:11]
    assert st["fp_sum"] == ref["fp_sum"][:11] and st["fp_xor"] == ref["fp_xor"][:11]
    assert st["peak_frontier_bytes"] <= 1 << 30
    pre = oracle.decide_prefix(adj, 10, 5, count_canonical=False)
    assert st["level_size"][:6] == pre["level_size"] and st["fp_sum"][:6] == pre["fp_sum"]


def test_out_of_core_level_keys_match_the_oracle():
    # a level written to host memory, downloaded set by set
    adj = gg.workload_gnp20()
    exp = oracle.level_keys(adj, 8, 6)
    with context(mem_cap_bytes=1 << 16, out_of_core=True) as ctx:
        r = ctx.decide_level(adj, k=8, level=6)
    assert np.array_equal(oracle.sort_keys(r["keys"]), exp)


# decide(6) of the n = 40 graph with 64 MB of device memory and 48 MB of host
# memory: levels 20 and 21 (46.9 MB and 45.8 MB of keys) fit neither memory
# alone next to each other, so at least one of them is split into a device
# part and a host part.
SPLIT_CAPS = dict(mem_cap_bytes=64 << 20, host_cap_mb=48, out_of_core=True)


def test_levels_split_between_device_and_host_match_the_golden_record():
    rec = json.load(open(os.path.join(GOLDEN, "rgg40_seed0_k6.json")))["decide"][0]
    adj = gg.workload_rgg40()
    with context(fingerprints=True, **SPLIT_CAPS) as ctx:
        r = ctx.decide(adj, k=6)
        st = r["stats"]
        assert r["yes"]
        assert st["level_size"] == rec["level_size"]
        assert st["fp_sum"] == [int(x) for x in rec["fp_sum"]]
        assert st["fp_xor"] == [int(x) for x in rec["fp_xor"]]
        assert st["generated"] == rec["canonical"]
        assert st["peak_frontier_bytes"] <= 64 << 20
    # the same device cap with too little host memory for the split is a
    # capacity error, not a wrong answer
    with context(mem_cap_bytes=64 << 20, host_cap_mb=8, out_of_core=True) as ctx:
        assert ctx.decide(adj, k=6, raise_on_error=False)["status"] == 2


@pytest.mark.parametrize("level", [20, 21])
def test_split_level_downloads_whole(level):
    # the peak levels downloaded set by set: the device part and the host part
    # together hold each set of the level once (size and digest of the
    # oracle's golden record)
    rec = json.load(open(os.path.join(GOLDEN, "rgg40_seed0_k6.json")))["decide"][0]
    adj = gg.workload_rgg40()
    with context(**SPLIT_CAPS) as ctx:
        r = ctx.decide_level(adj, k=6, level=level)
    keys = r["keys"].reshape(-1)
    assert r["count"] == rec["level_size"][level] == keys.size
    assert np.unique(keys).size == keys.size
    assert fingerprint_sums(keys) == (int(rec["fp_sum"][level]), int(rec["fp_xor"][level]))
