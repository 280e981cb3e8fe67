#!/usr/bin/env python
"""Benchmark: wavefront states expanded per second on one GB300.

Workload: the random geometric graph n=40, radius 0.25, seed 0 (64-bit
states), solved by the plain decide-at-k sweep from the minimum-degree /
minor-min-width lower bound to the exact treewidth, with elimination ordering
and tree decomposition output.  One step = one full ``tw_solve`` of that graph.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  ``value`` is states expanded per second with the
adjacency already resident in device memory (CUDA events on the library's
stream, L2 flushed before every step); ``e2e`` is the same metric through the
C ABI with host buffers.  ``roofline`` describes the expand+insert kernel: the
algorithmic bytes of its launches over their CUDA-event time.  ``cpu_baseline``
times the CPU oracle on a bounded sample of the same workload.
``--impl reference`` times the CPU oracle alone (the method's plain CPU form).
Under torchrun (N > 1) every rank solves its own replica of the graph (the
single-graph path does not shard); value = all ranks' states / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "wavefront states expanded/s"
UNIT = "states/s"
WORKLOAD = "random geometric graph n=40 r=0.25 seed 0; plain decide-at-k sweep from the lower bound to exact tw"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample length for cpu_baseline")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append(parts)
        os.remove(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ CPU baseline
def oracle_sample(seconds: float):
    """The CPU oracle as it stands on a bounded sample of the workload: the
    decide runs k = 0..5 of the same graph's plain sweep (the runs before the
    yes at tw = 6), repeated until `seconds` have passed."""
    import oracle
    from paper_1709_09990_gb300 import graphgen as gg
    adj = gg.workload_rgg40()
    states = 0
    runs = 0
    t0 = time.perf_counter()
    while True:
        for k in range(0, 6):
            states += oracle.decide(adj, k)["states_expanded"]
        runs += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": states / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle decide(k) for k=0..5 on the same graph, {runs} pass(es), {states} states in {dt:.1f} s"}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def expand_traffic():
    """Per-launch DRAM traffic of the expand kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "expand_insert_rgg40_traffic.json")))
    except (OSError, ValueError):
        return None
    src = open(os.path.join(ROOT, "paper_1709_09990_gb300", "csrc", "tw_expand.cu"), "rb").read()
    if rec.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import native

    stream = torch.cuda.Stream(device=dev)  # libtw runs on this stream; the events are recorded on it
    adj = gg.workload_rgg40()
    n = len(adj)
    rows_host = gg.to_rows_u64(adj).astype(np.int64)
    rows_dev = torch.from_numpy(rows_host).to(dev)
    tw_dev = torch.full((1,), -1, dtype=torch.int32, device=dev)
    order_dev = torch.full((n,), -1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    ctx = native.Context(device=local, stream=stream.cuda_stream, time_kernels=True)

    def step_device():
        return ctx.solve(rows_dev, n=n, tw_out=tw_dev, order_out=order_dev, want_td=True)

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    sampler = ClockSampler()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    torch.cuda.synchronize()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        res = step_device()
        ev[i][1].record(stream)
        stats.append(res["stats"])
    torch.cuda.synchronize()
    clocks = sampler.stop()
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    if world > 1:
        t = torch.tensor([dev_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_s = float(t.item())
        dist.barrier()
    tw = int(tw_dev.item())
    states_step = stats[-1]["states_expanded"]
    value = states_step * args.steps * world / dev_s

    # end to end through the C ABI with host buffers (pinned)
    rows_pin = torch.from_numpy(rows_host).pin_memory()
    tw_pin = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    order_pin = torch.full((n,), -1, dtype=torch.int32).pin_memory()
    parent_pin = torch.full((n,), -1, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_s = 0.0
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        native.lib().tw_solve(ctx._h, rows_pin.data_ptr(), n, tw_pin.data_ptr(), order_pin.data_ptr(),
                              parent_pin.data_ptr(), None, None)
        e2e_s += time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert int(tw_pin[0]) == tw

    st = stats[-1]
    pk = peaks()
    achieved = st["expand_bytes"] / st["expand_seconds"] / 1e9 if st["expand_seconds"] > 0 else None
    traffic = expand_traffic()
    roofline = None
    if achieved is not None:
        peak = pk["hbm_gbs"] if pk else 6800.0
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    "kernel": "expand_insert_kernel<uint64,4 warps>",
                    "peak_source": "measured" if pk else "fallback",
                    "bytes_per_launch": st["expand_bytes"] / max(1, st["expand_launches"]),
                    "launch_ms": 1e3 * st["expand_seconds"] / max(1, st["expand_launches"])}

    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * dev_s / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "tw": tw, "states_per_step": states_step,
                      "decide_runs_per_step": st["decide_runs"], "level_sizes": st["level_size"],
                      "peak_frontier_bytes": st["peak_frontier_bytes"], "l2": "flushed (512 MiB write) before each step",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "time_to_exact_tw_ms": round(1e3 * dev_s / args.steps, 3),
           "e2e": {"value": round(states_step * args.steps * world / e2e_s, 1), "unit": UNIT,
                   "h2d_bytes_per_step": int(rows_host.nbytes), "d2h_bytes_per_step": 4 + 8 * n,
                   "ms_per_step": round(1e3 * e2e_s / args.steps, 3)},
           "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
           "roofline": roofline, "clocks": clocks}
    ctx.close()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = oracle_sample(args.cpu_seconds)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle on rank 0: each step is the bounded oracle sample of the
    same workload (decide k = 0..5)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1709_09990_gb300 import graphgen as gg
    adj = gg.workload_rgg40()
    oracle.build()

    def step():
        s = 0
        for k in range(0, 6):
            s += oracle.decide(adj, k)["states_expanded"]
        return s

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    states = 0
    for _ in range(args.steps):
        states += step()
    dt = time.perf_counter() - t0
    value = states / dt
    sample = f"oracle decide(k) for k=0..5 of the workload graph per step ({states // max(1, args.steps)} states)"
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": len(adj)},
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
