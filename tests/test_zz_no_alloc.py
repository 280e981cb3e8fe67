"""tw_expand_level_static: one wavefront level with no device allocation.

The entry point exists for callers that cannot let a library allocate device
memory (a host that has handed the device's memory to its own pool, or a
latency-critical loop that cannot take cudaMalloc's device-wide
synchronisation).  Here the caller's buffers are torch tensors; the test chains
the entry point level by level from {empty set} and checks every level against
tw_decide (the allocating entry point) on two full runs in a row, so that the
second run starts from the scratch contents the first one left behind.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1709_09990_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

MAX_STATES = 1 << 20
M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix(z: np.ndarray) -> np.ndarray:
    # splitmix64 output function, wrapping uint64 arithmetic
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _fingerprints(keys: np.ndarray):
    f = _mix(keys.astype(np.uint64))
    with np.errstate(over="ignore"):
        s = int(np.sum(f, dtype=np.uint64))
    return s, int(np.bitwise_xor.reduce(f)) if f.size else 0


def _entry():
    from paper_1709_09990_gb300 import native
    lib = native.lib()
    f = lib.tw_expand_level_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                  ctypes.c_void_p]
    return f


def _chain(torch, f, adj, k, stream):
    """All levels 0 .. n-k-1 through the static entry point."""
    n = len(adj)
    dev = torch.device("cuda", 0)
    rows = torch.from_numpy(gg.to_rows_u64(adj).reshape(-1).astype(np.int64)).to(dev)
    cur = torch.zeros(1, dtype=torch.int64, device=dev)  # L_0 = {empty set}
    sizes, fps = [1], [(0, 0)]
    for i in range(0, n - k - 1):
        cap = min(MAX_STATES, max(64, cur.numel() * (n - i)))
        out = torch.empty(cap, dtype=torch.int64, device=dev)
        pred = torch.empty(cap, dtype=torch.uint8, device=dev)
        cnt = ctypes.c_uint64(0)
        rc = f(cur.data_ptr(), cur.numel(), rows.data_ptr(), n, k, out.data_ptr(), pred.data_ptr(), cap,
               ctypes.byref(cnt), stream.cuda_stream)
        assert rc == 0, rc
        m = int(cnt.value)
        keys = out[:m].cpu().numpy().view(np.uint64)
        pv = pred[:m].cpu().numpy().astype(np.uint64)
        # every output key holds its predecessor vertex and has i+1 vertices
        assert np.all((keys >> pv) & np.uint64(1) == 1)
        assert all(bin(int(x)).count("1") == i + 1 for x in keys[:2000])
        sizes.append(m)
        fps.append(_fingerprints(keys))
        if m == 0:
            break
        cur = out[:m].clone()
    return sizes, fps


@pytest.mark.parametrize("case", ["gnp20_k8", "gnp20_k7", "gnp44_k32", "rgg40_k5"])
def test_static_levels_match_tw_decide_twice(case):
    torch = pytest.importorskip("torch")
    from paper_1709_09990_gb300 import native
    graphs = {"gnp20_k8": (gg.workload_gnp20(), 8), "gnp20_k7": (gg.workload_gnp20(), 7),
              "gnp44_k32": (gg.gnp(44, 0.5, 4), 32), "rgg40_k5": (gg.workload_rgg40(), 5)}
    adj, k = graphs[case]
    with native.Context(device=0, fingerprints=True) as ctx:
        ref = ctx.decide(adj, k=k)["stats"]
    f = _entry()
    stream = torch.cuda.Stream(device=0)
    for _ in range(2):  # two calls in a row over the same static scratch
        sizes, fps = _chain(torch, f, adj, k, stream)
        assert sizes == ref["level_size"]
        assert [s for s, _ in fps] == ref["fp_sum"]
        assert [x for _, x in fps] == ref["fp_xor"]


def test_static_limits_are_reported():
    torch = pytest.importorskip("torch")
    f = _entry()
    adj = gg.workload_gnp20()
    dev = torch.device("cuda", 0)
    rows = torch.from_numpy(gg.to_rows_u64(adj).reshape(-1).astype(np.int64)).to(dev)
    start = torch.zeros(1, dtype=torch.int64, device=dev)
    out = torch.empty(64, dtype=torch.int64, device=dev)
    pred = torch.empty(64, dtype=torch.uint8, device=dev)
    cnt = ctypes.c_uint64(0)
    stream = torch.cuda.Stream(device=0)
    # a capacity above the fixed table's limit is refused before any work
    rc = f(start.data_ptr(), 1, rows.data_ptr(), 20, 8, out.data_ptr(), pred.data_ptr(), MAX_STATES + 1,
           ctypes.byref(cnt), stream.cuda_stream)
    assert rc == 1
    # an output buffer smaller than the level: capacity status and the true count
    rc = f(start.data_ptr(), 1, rows.data_ptr(), 20, 8, out.data_ptr(), pred.data_ptr(), 3,
           ctypes.byref(cnt), stream.cuda_stream)
    assert rc == 2 and int(cnt.value) == 18


def test_static_small_buffer_still_counts_exactly_and_rejects_the_full_set():
    torch = pytest.importorskip("torch")
    from paper_1709_09990_gb300 import native
    f = _entry()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=0)
    adj = gg.workload_gnp20()
    rows = torch.from_numpy(gg.to_rows_u64(adj).reshape(-1).astype(np.int64)).to(dev)
    with native.Context(device=0) as ctx:
        lvl3 = ctx.decide_level(adj, k=8, level=3)["keys"]
        n4 = ctx.decide_level(adj, k=8, level=4)["count"]
    assert n4 > 1024  # more states than the table a 3-state buffer is given
    inp = torch.from_numpy(lvl3.reshape(-1).astype(np.int64)).to(dev)
    out = torch.empty(64, dtype=torch.int64, device=dev)
    pred = torch.empty(64, dtype=torch.uint8, device=dev)
    cnt = ctypes.c_uint64(0)
    rc = f(inp.data_ptr(), inp.numel(), rows.data_ptr(), 20, 8, out.data_ptr(), pred.data_ptr(), 3,
           ctypes.byref(cnt), stream.cuda_stream)
    assert rc == 2 and int(cnt.value) == n4
    # n = 64: a 63-vertex input set would extend to the all-ones set, the
    # table's empty marker, so the call is refused
    path = gg.path(64)
    prow = torch.from_numpy(gg.to_rows_u64(path).reshape(-1).astype(np.int64)).to(dev)
    big = torch.tensor([np.int64(-2)], dtype=torch.int64, device=dev)  # every vertex but 0
    rc = f(big.data_ptr(), 1, prow.data_ptr(), 64, 1, out.data_ptr(), pred.data_ptr(), 64,
           ctypes.byref(cnt), stream.cuda_stream)
    assert rc == 1
