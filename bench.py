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
    ap.add_argument("--workload", default="rgg40", choices=["rgg40", "gnp20", "pktree60", "batch", "learned"],
                    help="rgg40 (default): the n=40 geometric graph; gnp20: G(20,0.3); pktree60: the partial "
                         "10-tree n=60 at k=10; batch: the 4096-graph batch vs a per-graph loop; learned: the "
                         "learned starting bound vs the plain sweep")
    ap.add_argument("--graphs", type=int, default=0, help="batch/learned: number of graphs (0 = full workload)")
    ap.add_argument("--triage-cap-gb", type=float, default=0.5,
                    help="batch/learned: device cap of the per-graph loop that sorts out the heavy graphs")
    ap.add_argument("--heavy", action="store_true", help="batch: also solve the heavy graphs (default cap)")
    ap.add_argument("--arena-sweep", action="store_true",
                    help="batch: also time the persistent kernel with smaller block arenas")
    ap.add_argument("--mem-cap-gb", type=float, default=0.0, help="device memory cap per context (0 = default)")
    ap.add_argument("--spill-levels", action="store_true",
                    help="keep finished levels in pinned host memory (tw_config.spill_levels)")
    ap.add_argument("--no-sub", action="store_true", help="skip the other workloads' sub-records")
    ap.add_argument("--in-core", action="store_true", help="pktree60: no out-of-core levels (stop at the cap)")
    ap.add_argument("--host-cap-gb", type=float, default=0.0,
                    help="pktree60: pinned host memory for out-of-core levels (0 = 80%% of the memory this "
                         "process may use: MemAvailable, or the cgroup limit when lower)")
    ap.add_argument("--plain", action="store_true", help="pktree60: without the clique skip")
    ap.add_argument("--partition-mb", type=int, default=0,
                    help="tw_config.partition_table_mb (0 = library default, -1 = never, -2 = every level)")
    ap.add_argument("--graph-levels", type=int, default=0, help="tw_config.graph_levels (pktree60, gnp20)")
    ap.add_argument("--fused-off", action="store_true", help="gnp20: the level loop instead of the fused launch")
    ap.add_argument("--ncu-record", nargs=2, metavar=("CSV", "FIRST_LEVEL"),
                    help="write profiles/expand_insert_rgg40_counters.json from an ncu CSV of consecutive "
                         "expand launches starting at FIRST_LEVEL, then exit")
    ap.add_argument("--ncu-command", default="", help="the ncu command line recorded with --ncu-record")
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


# ------------------------------------------------------------- multi-rank
def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / slowest_seconds


# ------------------------------------------------------------ CPU baseline
# The timed GPU step is one tw_solve of the n=40 geometric graph: its lower
# bound is already tw = 6, so the step is the single decide run at k = 6
# (79,399,414 states).  The oracle cannot finish that run in a bounded sample,
# so its sample is the start of the same run: decide(6) up to level 8, i.e.
# the expansion of levels 0 .. 7 (304,654 states), repeated.
ORACLE_K = 6
ORACLE_LEVELS = 8


def oracle_step():
    """One bounded oracle sample: levels 0 .. ORACLE_LEVELS of decide(6) of the
    benchmark graph; returns the states it expanded."""
    import oracle
    from paper_1709_09990_gb300 import graphgen as gg
    return oracle.decide_prefix(gg.workload_rgg40(), ORACLE_K, ORACLE_LEVELS, count_canonical=False)["states_expanded"]


def oracle_sample(seconds: float):
    """The CPU oracle as it stands, timed on the host for at least `seconds`
    over repeats of :func:`oracle_step`."""
    states = 0
    runs = 0
    t0 = time.perf_counter()
    while True:
        states += oracle_step()
        runs += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": states / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the first {ORACLE_LEVELS} levels of the same decide run (k={ORACLE_K}; {states // runs} of its "
                      f"79,399,414 states) on one host core, {runs} repeat(s), {states} states in {dt:.1f} s"}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def kernel_source_hash() -> str:
    """sha256 of the expand kernel's sources with comments and blank space
    removed (a comment edit does not change the kernel)."""
    import re
    csrc = os.path.join(ROOT, "paper_1709_09990_gb300", "csrc")
    code = []
    for f in ("tw_expand.cu", "tw_expand_core.cuh", "tw_keys.cuh", "tw_internal.h"):
        src = open(os.path.join(csrc, f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        code.append(" ".join(src.split()))
    return hashlib.sha256("\n".join(code).encode()).hexdigest()


COUNTERS = os.path.join(ROOT, "profiles", "expand_insert_rgg40_counters.json")


def expand_counters():
    """The committed ncu counters of a few expand launches of the benchmark
    step (see write_counter_record), or None when the kernel source changed
    since they were taken."""
    try:
        rec = json.load(open(COUNTERS))
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_hash():
        return None
    return rec


def write_counter_record(csv_path: str, first_level: int, command: str) -> dict:
    """Turns the ncu CSV of consecutive expand launches (levels first_level,
    first_level + 1, ... of the benchmark's decide run) into the counter
    record the bench reads: per launch DRAM bytes, ALU-pipe and total warp
    instructions, duration, and the ALU pipe's peak rate."""
    import csv
    by_id, names = {}, set()
    for row in csv.DictReader(l for l in open(csv_path) if l.startswith('"')):
        if "expand" not in row.get("Kernel Name", ""):
            continue
        names.add(row["Kernel Name"])
        v = row["Metric Value"].replace(",", "")
        by_id.setdefault(int(row["ID"]), {})[row["Metric Name"]] = float(v)
    launches = [by_id[i] for i in sorted(by_id)]
    rec = {"kernel": " / ".join(sorted(names)),
           "workload": "random geometric graph n=40 r=0.25 seed 0, decide(6) of one tw_solve",
           "levels": [first_level + j for j in range(len(launches))],
           "dram_bytes": [m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"] for m in launches],
           "alu_warp_inst": [m["sm__inst_executed_pipe_alu.sum"] for m in launches],
           "warp_inst": [m["smsp__inst_executed.sum"] for m in launches],
           "duration_ns": [m["gpu__time_duration.sum"] for m in launches],
           "alu_pct_of_peak": [m["sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active"] for m in launches],
           "alu_peak_warp_inst_per_sm_cycle": launches[0]["sm__inst_executed_pipe_alu.avg.peak_sustained"],
           "source_sha256": kernel_source_hash(), "command": command,
           "scaling": "per input state: the step's launches are credited with the captured launches' "
                      "counts per input state times their own input states"}
    with open(COUNTERS, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def roofline_of(st, pk, clocks):
    """The expand kernel's rooflines for one step's statistics: ALU pipe (the
    bound its profile shows on this L2-resident workload) and HBM."""
    if not st["expand_seconds"]:
        return None
    launches = max(1, st["expand_launches"])
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    hbm_achieved = st["expand_bytes"] / st["expand_seconds"] / 1e9
    out = {"kernel": "the expand+insert kernel (core::expand_level; graph_expand_kernel<uint64, 4 warps> in the "
                     "graph-driven level loop the step runs)",
           "launch_ms": 1e3 * st["expand_seconds"] / launches,
           "bytes_per_launch": st["expand_bytes"] / launches,
           "hbm": {"achieved": round(hbm_achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                   "frac": round(hbm_achieved / hbm_peak, 4), "peak_source": "measured" if pk else "fallback"}}
    rec = expand_counters()
    traffic = None
    if rec:
        sizes = st["level_size"]
        cap_states = sum(sizes[i] for i in rec["levels"])
        per_state = lambda xs: sum(xs) / cap_states  # noqa: E731
        traffic = per_state(rec["dram_bytes"]) * st["states_expanded"] / launches
        alu_inst = per_state(rec["alu_warp_inst"]) * st["states_expanded"]
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        sms = 152
        alu_peak = rec["alu_peak_warp_inst_per_sm_cycle"] * sms * sm_mhz * 1e6 / 1e9
        alu_achieved = alu_inst / st["expand_seconds"] / 1e9
        out.update({"bound": "alu", "achieved": round(alu_achieved, 1), "peak": round(alu_peak, 1),
                    "unit": "G ALU-pipe warp-instructions/s", "frac": round(alu_achieved / alu_peak, 4),
                    "traffic": round(traffic, 1),
                    "alu_frac": round(alu_achieved / alu_peak, 4),
                    "alu_frac_ncu_captured": [round(x / 100.0, 4) for x in rec["alu_pct_of_peak"]],
                    "peak_note": f"{rec['alu_peak_warp_inst_per_sm_cycle']} ALU warp-instructions per SM cycle "
                                 f"(ncu peak_sustained) x {sms} SMs x {sm_mhz:.0f} MHz (median SM clock under load)",
                    "counters_from": f"ncu, levels {rec['levels']} of the step, scaled per input state"})
    else:
        out.update({"bound": "hbm", "achieved": round(hbm_achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(hbm_achieved / hbm_peak, 4), "traffic": None})
    out["hbm"]["traffic_over_algorithmic"] = round(traffic / out["bytes_per_launch"], 3) if traffic else None
    return out


# ------------------------------------------------------ other workloads
def sub_gnp20(stream, steps):
    """G(20, 0.3) seed 0 (32-bit states): the plain sweep from the lower bound
    with ordering and tree decomposition; CUDA events on libtw's stream."""
    import numpy as np
    import torch
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import native
    adj = gg.workload_gnp20()
    rows = torch.from_numpy(gg.to_rows_u64(adj).astype(np.int64)).cuda()
    with native.Context(device=torch.cuda.current_device(), stream=stream.cuda_stream) as ctx:
        for _ in range(3):
            res = ctx.solve(rows, n=20, want_td=True)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches = 0
        for a, b in ev:
            a.record(stream)
            res = ctx.solve(rows, n=20, want_td=True)
            b.record(stream)
            launches += res["stats"]["kernel_launches"]
        torch.cuda.synchronize()
    dt = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    st = res["stats"]
    return {"workload": "G(n=20, p=0.3) seed 0; plain sweep from the lower bound to exact tw, ordering + tree "
                        "decomposition", "dtype": "u32", "tw": res["tw"], "metric": METRIC,
            "value": round(st["states_expanded"] * steps / dt, 1), "unit": UNIT,
            "time_to_exact_tw_ms": round(1e3 * dt / steps, 4), "states_per_solve": st["states_expanded"],
            "decide_runs": st["decide_runs"], "gpu_launches_per_solve": launches // steps,
            "level_sizes_final_k": st["level_size"], "steps": steps}


def sub_pktree60(args):
    """The partial 10-tree n=60 seed 0 at k = 10 under the default cap
    (150 GB or 90% of free memory): the levels reached, with the Section 3.1
    clique skip on (it shrinks this graph's wavefront) and off."""
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import native
    adj = gg.workload_pktree60()
    out = {"workload": "partial 10-tree n=60 (30% of edges removed) seed 0; decide at k=10", "dtype": "u64"}
    for name, kw in (("plain", {}), ("clique_skip", {"clique_skip": True})):
        with native.Context(device=0, time_kernels=True, **kw) as ctx:
            b = ctx.bounds(adj).tolist()
            t = time.perf_counter()
            r = ctx.decide(adj, k=10, raise_on_error=False)
            dt = time.perf_counter() - t
        st = r["stats"]
        out[name] = {"status": native.strerror(r["status"]), "yes": r["yes"] if r["status"] == 0 else None,
                     "seconds": round(dt, 3), "levels_reached": st["level_size"],
                     "states_expanded": st["states_expanded"], "states_per_s": round(st["states_expanded"] / dt, 1),
                     "peak_frontier_bytes": st["peak_frontier_bytes"],
                     "expand_algorithmic_GBps": round(st["expand_bytes"] / st["expand_seconds"] / 1e9, 1)
                     if st["expand_seconds"] else None}
        out["bounds"] = {"mmd": b[0], "mmd_plus": b[1], "min_degree_width": b[2], "min_fill_width": b[3]}
        out["tw_from_bounds"] = b[1] if max(b[0], b[1]) == min(b[2], b[3]) else None
    return out


def sub_batch(args, count=512):
    """The first `count` graphs of the 4096-graph batch workload: the light
    ones (solved by the per-graph loop within 2^21 states under the triage
    cap) through the persistent batched kernel, the level-synchronous one and
    the per-graph loop."""
    from paper_1709_09990_gb300 import graphgen as gg
    graphs = gg.batch_graphs(count)
    light, loop_tw, _, loop_secs = batch_light(graphs, int(args.triage_cap_gb * (1 << 30)))
    rec = batch_arms(graphs, light, loop_tw, loop_secs)
    return {"workload": f"the first {count} graphs of the 4096-graph batch workload (seeds 0..{count - 1}), the "
                        f"light ones (solved within {LIGHT_STATES} states)", "dtype": "u32/u64",
            "heavy_graphs": count - len(light), **rec}


def sub_learned(args, ntr=2000, nte=200):
    """A small sample of the learned-k workload: train on `ntr` graphs with n
    in [12, 40], compare on `nte` held-out graphs with n in [30, 56] (those the
    per-graph loop solves under the triage cap)."""
    rec = learned_compare(ntr, nte, int(args.triage_cap_gb * (1 << 30)))
    rec["workload"] = (f"learned-k sample: train {ntr} graphs n in [12,40] (seeds 1e6+j), test {nte} graphs n in "
                       "[30,56] (seeds 2e6+j); the full config is --workload learned")
    return rec


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

    ctx = native.Context(device=local, stream=stream.cuda_stream, time_kernels=True,
                         spill_levels=args.spill_levels)

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
    dev_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dev)
    if world > 1:
        dist.barrier()
    tw = int(tw_dev.item())
    states_step = stats[-1]["states_expanded"]
    value = job_throughput(states_step * args.steps, world, dev_s)

    # end to end through the C ABI with host buffers (pinned), the same
    # outputs as the device step: tw, ordering, tree decomposition
    words = max(1, (n + 63) // 64)
    rows_pin = torch.from_numpy(rows_host).pin_memory()
    tw_pin = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    order_pin = torch.full((n,), -1, dtype=torch.int32).pin_memory()
    parent_pin = torch.full((n,), -1, dtype=torch.int32).pin_memory()
    bags_pin = torch.zeros((n, words), dtype=torch.int64).pin_memory()
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
                              parent_pin.data_ptr(), bags_pin.data_ptr(), None)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dev)
    assert int(tw_pin[0]) == tw

    st = stats[-1]
    roofline = roofline_of(st, peaks(), clocks)
    d2h = tw_pin.nbytes + order_pin.nbytes + parent_pin.nbytes + bags_pin.nbytes

    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * dev_s / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "tw": tw, "states_per_step": states_step,
                      "decide_runs_per_step": st["decide_runs"], "level_sizes": st["level_size"],
                      "peak_frontier_bytes": st["peak_frontier_bytes"], "l2": "flushed (512 MiB write) before each step",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "time_to_exact_tw_ms": round(1e3 * dev_s / args.steps, 3),
           "e2e": {"value": round(job_throughput(states_step * args.steps, world, e2e_s), 1), "unit": UNIT,
                   "h2d_bytes_per_step": int(rows_host.nbytes), "d2h_bytes_per_step": int(d2h),
                   "ms_per_step": round(1e3 * e2e_s / args.steps, 3),
                   "outputs": "tw, ordering, tree decomposition (parents and bags), as in the device-timed step"},
           "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
           "roofline": roofline, "clocks": clocks}
    if world == 1 and not args.no_sub:
        # the other workloads, after the timed region
        out["other_workloads"] = {}
        for name, fn in (("gnp20", lambda: sub_gnp20(stream, max(5, args.steps))),
                         ("pktree60", lambda: sub_pktree60(args)), ("batch", lambda: sub_batch(args)),
                         ("learned", lambda: sub_learned(args))):
            try:
                out["other_workloads"][name] = fn()
            except Exception as e:  # a failed sub-record must not hide the main line
                out["other_workloads"][name] = {"error": f"{type(e).__name__}: {e}"}
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
    same workload (the first levels of the same decide run)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1709_09990_gb300 import graphgen as gg
    adj = gg.workload_rgg40()
    oracle.build()
    step = oracle_step

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    states = 0
    for _ in range(args.steps):
        states += step()
    dt = time.perf_counter() - t0
    value = states / dt
    sample = (f"oracle: the first {ORACLE_LEVELS} levels of the benchmark step's decide run (k={ORACLE_K}; "
              f"{states // max(1, args.steps)} of its 79,399,414 states) per step, one host core")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": len(adj)},
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ other workloads
def _line(metric, value, unit, args, config, extra):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": unit.endswith("/s"), "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "config": config}
    out.update(extra)
    print(json.dumps(out), flush=True)


def run_gnp20(args):
    """G(20, 0.3) seed 0, 32-bit states: the sweep from the lower bound (k = 6,
    7, 8) with ordering and tree decomposition, by default in one fused launch
    (--fused-off runs the level loop instead)."""
    import numpy as np
    import torch
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import native
    adj = gg.workload_gnp20()
    stream = torch.cuda.Stream()
    ctx = native.Context(device=0, stream=stream.cuda_stream, fused_states=-1 if args.fused_off else 0,
                         graph_levels=args.graph_levels)
    rows = torch.from_numpy(gg.to_rows_u64(adj).astype(np.int64)).cuda()
    for _ in range(args.warmup):
        ctx.solve(rows, n=20, want_td=True)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record(stream)
        res = ctx.solve(rows, n=20, want_td=True)
        b.record(stream)
    torch.cuda.synchronize()
    dt = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    st = res["stats"]
    _line(METRIC, round(st["states_expanded"] * args.steps / dt, 1), UNIT, args,
          {"workload": "G(n=20, p=0.3) seed 0; plain sweep from the lower bound to exact tw", "n": 20, "tw": res["tw"],
           "states_per_step": st["states_expanded"], "decide_runs_per_step": st["decide_runs"],
           "level_sizes_final_k": st["level_size"]},
          {"ms_per_step": round(1e3 * dt / args.steps, 4), "time_to_exact_tw_ms": round(1e3 * dt / args.steps, 4),
           "gpu_launches": st["kernel_launches"] * args.steps, "dtype": "u32"})
    ctx.close()


def host_cap_mb(args) -> int:
    """Pinned host memory (MB) the out-of-core levels may take: --host-cap-gb,
    else 80% of what this process may use (MemAvailable, or the cgroup's
    memory limit minus its current use when that is lower)."""
    if args.host_cap_gb:
        return int(args.host_cap_gb * 1024)
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for lim, cur in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                     ("/sys/fs/cgroup/memory/memory.limit_in_bytes", "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            v = open(lim).read().strip()
            if v.isdigit() and int(v) < (1 << 60):
                room = int(v) - int(open(cur).read().strip())
                avail = room if avail is None else min(avail, room)
        except (OSError, ValueError):
            pass
    return int(0.80 * avail) >> 20 if avail else 0


def run_pktree60(args):
    """Partial 10-tree n=60 seed 0: decide at k = 10 (the lower bound MMD+ =
    10 certifies no at k = 9) with the Section 3.1 clique skip and out-of-core
    levels: the table is built in hash-range slices that fit the device cap and
    levels that do not fit the device go to host memory.  Reports the answer,
    every level size, states/s and the device bytes used."""
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import native
    adj = gg.workload_pktree60()
    cap = int(args.mem_cap_gb * (1 << 30)) if args.mem_cap_gb else 150 << 30
    hcap = host_cap_mb(args)
    with native.Context(device=0, mem_cap_bytes=cap, time_kernels=True, clique_skip=not args.plain,
                        out_of_core=not args.in_core, partition_table_mb=args.partition_mb,
                        graph_levels=args.graph_levels, host_cap_mb=hcap) as ctx:
        b = ctx.bounds(adj).tolist()
        t = time.perf_counter()
        r = ctx.decide(adj, k=10, raise_on_error=False)
        dt = time.perf_counter() - t
    st = r["stats"]
    answered = r["status"] == 0
    _line(METRIC, round(st["states_expanded"] / dt, 1), UNIT, args,
          {"workload": "partial 10-tree n=60 (30% of edges removed) seed 0; decide at k=10"
                       + ("" if args.plain else " with the clique skip"),
           "n": 60, "bounds": {"mmd": b[0], "mmd_plus": b[1], "min_degree_width": b[2], "min_fill_width": b[3]},
           "mem_cap_gb": round(cap / (1 << 30), 1), "out_of_core": not args.in_core,
           "host_cap_gb": round(hcap / 1024, 1),
           "partition_table_mb": args.partition_mb},
          {"status": native.strerror(r["status"]), "status_code": r["status"],
           "yes": r["yes"] if answered else None,
           "tw": 10 if answered and r["yes"] and max(b[0], b[1]) == 10 else None,
           "seconds": round(dt, 3), "time_to_exact_tw_s": round(dt, 3) if answered else None,
           "levels": st["level_size"], "states_expanded": st["states_expanded"],
           "generated_pairs": st["generated"], "expand_launches": st["expand_launches"],
           "peak_device_bytes": st["peak_frontier_bytes"],
           "expand_algorithmic_GBps": round(st["expand_bytes"] / st["expand_seconds"] / 1e9, 1)
           if st["expand_seconds"] else None})


def triage_loop(graphs, cap_bytes):
    """The plain per-graph loop (tw_solve with ordering) under a small device
    cap: graphs whose sweep fits it solve exactly as under any larger cap (the
    same fused launch or level loop), the others stop at the cap quickly with
    TW_ERR_CAPACITY.  Returns per-graph tw (-1 over the cap), states and
    seconds."""
    from paper_1709_09990_gb300 import native
    tw, states, secs = [], [], []
    with native.Context(device=0, mem_cap_bytes=cap_bytes) as ctx:
        for a in graphs[:16]:
            try:
                ctx.solve(a, want_order=True)
            except native.TwError:
                pass
        for a in graphs:
            t = time.perf_counter()
            try:
                r = ctx.solve(a, want_order=True)
                tw.append(r["tw"])
                states.append(r["stats"]["states_expanded"])
            except native.TwError:
                tw.append(-1)
                states.append(-1)
            secs.append(time.perf_counter() - t)
    return tw, states, secs


def batch_light(graphs, triage_cap, light_states=None):
    """Light graphs of a set (the per-graph loop solves them under the triage
    cap within light_states states): their indices, loop answers and loop
    time, and the number of heavy graphs."""
    light_states = light_states or LIGHT_STATES
    tw, states, secs = triage_loop(graphs, triage_cap)
    light = [i for i in range(len(graphs)) if tw[i] >= 0 and states[i] <= light_states]
    return light, tw, states, secs


def batch_arms(graphs, light, loop_tw, loop_secs):
    """The persistent batched kernel (one launch for all light graphs) and the
    level-synchronous batched kernel on the light graphs, against the loop's
    time on the same graphs; default device cap."""
    from paper_1709_09990_gb300 import native
    sub = [graphs[i] for i in light]
    rec = {"graphs": len(sub), "loop_seconds": round(sum(loop_secs[i] for i in light), 4)}
    with native.Context(device=0) as ctx, native.Context(device=0, batch_kernel=1) as sync:
        ctx.solve_batch(sub[:64])
        sync.solve_batch(sub[:64])
        for arm, c in (("persistent", ctx), ("level_synchronous", sync)):
            t = time.perf_counter()
            res = c.solve_batch(sub)
            dt = time.perf_counter() - t
            ok = res["per_graph_status"] == 0
            rec[arm] = {"seconds": round(dt, 4), "solved": int(ok.sum()),
                        "same_answers_as_loop": bool(all(int(res["tw"][j]) == loop_tw[i]
                                                         for j, i in enumerate(light) if ok[j])),
                        "kernel_launches": res["stats"]["kernel_launches"],
                        "states_per_s": round(res["stats"]["states_expanded"] / dt, 1) if dt else None,
                        "speedup_vs_loop": round(rec["loop_seconds"] / dt, 3) if dt else None}
    return rec


def run_batch(args):
    """The 4096-graph batch (G(n,p) and partial k-trees, n in [16, 48]).
    Graphs are first sorted by the per-graph loop (tw_solve with ordering)
    under a small device cap (--triage-cap-gb): the light ones (solved within
    2^21 states) are the ones the batch design is for; on them the persistent
    batched kernel (one launch) and the level-synchronous batched kernel run
    against the loop's time.  Heavy graphs leave the batch for the
    single-graph path in every arm, so they measure that path, not the batch;
    they are counted, and solved here only with --heavy (default cap)."""
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import native
    N = args.graphs or 4096
    graphs = gg.batch_graphs(N)
    t = time.perf_counter()
    light, loop_tw, loop_states, loop_secs = batch_light(graphs, int(args.triage_cap_gb * (1 << 30)))
    triage_s = time.perf_counter() - t
    rec = batch_arms(graphs, light, loop_tw, loop_secs)
    if args.arena_sweep:
        # the persistent kernel with smaller block arenas: graphs that outgrow
        # one continue in the level-synchronous kernel
        sub = [graphs[i] for i in light]
        rec["persistent_by_arena_states"] = {}
        for A in (1 << 19, 1 << 17, 1 << 15, 1 << 13):
            with native.Context(device=0, batch_arena_states=A) as c:
                c.solve_batch(sub[:64])
                t = time.perf_counter()
                res = c.solve_batch(sub)
                dt = time.perf_counter() - t
            rec["persistent_by_arena_states"][str(A)] = {
                "seconds": round(dt, 4), "kernel_launches": res["stats"]["kernel_launches"],
                "same_answers_as_loop": bool(all(int(res["tw"][j]) == loop_tw[i] for j, i in enumerate(light)))}
    heavy = [i for i in range(N) if i not in set(light)]
    out = {"light": rec, "heavy_graphs": len(heavy),
           "heavy_over_triage_cap": sum(1 for i in heavy if loop_tw[i] < 0),
           "triage_seconds": round(triage_s, 3)}
    if args.heavy:
        with native.Context(device=0) as ctx:
            t = time.perf_counter()
            res = ctx.solve_batch([graphs[i] for i in heavy])
            out["heavy"] = {"seconds": round(time.perf_counter() - t, 3),
                            "solved": int((res["per_graph_status"] == 0).sum())}
    _line("time to exact tw, batch (light graphs)", rec["persistent"]["seconds"], "s", args,
          {"workload": f"{N} seeded graphs: even seeds G(n,p), n~U{{16..48}}, p~U[0.1,0.5]; odd seeds partial "
                       "k-trees, k~U{3..12}, 30% edges removed", "graphs": N,
           "light_states_limit": LIGHT_STATES, "triage_cap_gb": args.triage_cap_gb},
          out)


LIGHT_STATES = 1 << 21  # states per solve below which a graph counts as light in the batch report


def learned_compare(ntr, nte, tcap):
    """Label ntr training graphs (batched solve under the triage cap), train
    the network on the device, then solve the held-out graphs that the
    per-graph loop solves under that cap with proposals (batched) and with the
    plain sweep (batched and the loop's own time)."""
    import numpy as np
    from paper_1709_09990_gb300 import graphgen as gg
    from paper_1709_09990_gb300 import learned
    from paper_1709_09990_gb300 import native
    tr = [gg.mixed_graph(10**6 + j, 12, 40, j % 2 == 0) for j in range(ntr)]
    te = [gg.mixed_graph(2 * 10**6 + j, 30, 56, j % 2 == 0) for j in range(nte)]
    with native.Context(device=0, mem_cap_bytes=tcap) as small:
        L = learned.label(small, tr)
    ok = L["status"] == 0
    t = time.perf_counter()
    loop_tw, loop_states, loop_secs = triage_loop(te, tcap)
    loop_all_s = time.perf_counter() - t
    solved = [i for i in range(nte) if loop_tw[i] >= 0]
    sub = [te[i] for i in solved]
    with native.Context(device=0) as ctx:
        # offset chosen on a validation split of the training graphs
        idx = np.arange(len(tr))[ok]
        val = idx[idx % 10 == 0]
        fit = idx[idx % 10 != 0]
        t = time.perf_counter()
        T = learned.train(ctx, L["x"][fit], L["tw"][fit], L["n"][fit], epochs=60)
        train_s = time.perf_counter() - t
        lbv = np.array([max(ctx.bounds(tr[i])[:2]) for i in val])
        pv = learned.propose(ctx, T["params"], L["x"][val], L["n"][val])
        off = learned.choose_offset(pv, L["tw"][val], lbv)
        n = np.array([len(g) for g in sub], np.int32)
        ctx.solve_batch(sub[:32])
        t = time.perf_counter()
        hint = learned.propose(ctx, T["params"], ctx.features(sub), n, off)
        lk = ctx.solve_batch(sub, k_hint=hint)
        t_learned = time.perf_counter() - t
        t = time.perf_counter()
        pb = ctx.solve_batch(sub)
        t_plain_batch = time.perf_counter() - t
    okl = lk["per_graph_status"] == 0
    ref = np.array([loop_tw[i] for i in solved])
    t_loop = sum(loop_secs[i] for i in solved)
    return {"learned_batch_seconds": round(t_learned, 4), "label_seconds": round(L["seconds"], 2),
            "train_seconds": round(train_s, 3), "train_graphs_used": int(ok.sum()),
            "final_train_loss": float(T["loss"][-1]), "offset": off,
            "test_graphs_compared": len(solved), "test_over_triage_cap": nte - len(solved),
            "test_solved_learned": int(okl.sum()),
            "exact_answer_rate": float((lk["tw"][okl] == ref[okl]).mean()) if okl.any() else None,
            "plain_batch_same_answers": bool((pb["tw"] == ref).all()),
            "proposal_hits_tw": float((np.rint(hint) == ref).mean()) if len(ref) else None,
            "plain_loop_seconds": round(t_loop, 4), "plain_batch_seconds": round(t_plain_batch, 4),
            "speedup_vs_plain_loop": round(t_loop / t_learned, 3) if t_learned else None,
            "loop_seconds_with_triaged_out_graphs": round(loop_all_s, 3),
            "decide_runs": {"learned_batch": lk["stats"]["decide_runs"], "plain_batch": pb["stats"]["decide_runs"]}}


def run_learned(args):
    """Learned starting bound: label and train on the 20000 training graphs
    (n in [12, 40]), then solve the 2000 held-out graphs (n in [30, 56]) with
    proposals (batched) and with the plain per-graph sweep.  Labels come from
    the batched solve under the triage cap (graphs over it are left out of
    training); the held-out graphs are sorted by the per-graph loop under the
    same cap, and the arms are compared on the ones it solves (default cap for
    the batched arms)."""
    ntr = args.graphs * 10 if args.graphs else 20000
    nte = args.graphs or 2000
    rec = learned_compare(ntr, nte, int(args.triage_cap_gb * (1 << 30)))
    _line("time to exact tw, learned-k batched", rec.pop("learned_batch_seconds"), "s", args,
          {"workload": f"train {ntr} graphs n in [12,40] (seeds 1e6+j), test {nte} graphs n in [30,56] "
                       "(seeds 2e6+j), mixed G(n,p) / partial k-trees", "triage_cap_gb": args.triage_cap_gb},
          rec)


def main():
    args = parse()
    if args.ncu_record:
        print(json.dumps(write_counter_record(args.ncu_record[0], int(args.ncu_record[1]), args.ncu_command)))
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "rgg40":
        run_ours(args)
    else:
        {"gnp20": run_gnp20, "pktree60": run_pktree60, "batch": run_batch, "learned": run_learned}[args.workload](args)


if __name__ == "__main__":
    main()
