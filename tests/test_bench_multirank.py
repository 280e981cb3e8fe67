"""bench.py's N > 1 path on CPU: two gloo ranks agree on the slowest rank's
time and on the whole-job rate (the GPU runs use the same helpers over NCCL)."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.max_over_ranks(1.5 + rank, "cpu")  # rank 1 is slower
    rate = bench.job_throughput(1000.0, dist.get_world_size(), slowest)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["slowest"] == 2.5
        assert r["rate"] == pytest.approx(2 * 1000.0 / 2.5)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    assert bench.job_throughput(10.0, 1, 2.0) == 5.0


def test_host_cap_for_out_of_core_runs():
    # an explicit --host-cap-gb wins; otherwise 80% of what the process may
    # use (MemAvailable, or the cgroup limit when lower), in MB
    import argparse
    import bench
    assert bench.host_cap_mb(argparse.Namespace(host_cap_gb=2.5)) == 2560
    got = bench.host_cap_mb(argparse.Namespace(host_cap_gb=0.0))
    avail = None
    for line in open("/proc/meminfo"):
        if line.startswith("MemAvailable:"):
            avail = int(line.split()[1]) * 1024
    if avail:
        assert 0 < got <= int(0.80 * avail) >> 20
