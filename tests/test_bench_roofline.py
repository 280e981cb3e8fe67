"""bench.py's roofline arithmetic on CPU: the expand kernel's HBM and ALU-pipe
figures from a step's statistics and an ncu counter record, and the parser that
turns an ncu CSV of consecutive expand launches into that record."""
import json

import pytest

import bench


def _stats():
    # three levels of 100, 200 and 300 input states; 6 launches in all
    return {"expand_seconds": 2e-3, "expand_launches": 6, "expand_bytes": 12e6,
            "level_size": [1, 100, 200, 300, 50], "states_expanded": 600}


def test_hbm_roofline_without_counters(monkeypatch):
    monkeypatch.setattr(bench, "expand_counters", lambda: None)
    r = bench.roofline_of(_stats(), {"hbm_gbs": 6000.0}, {"sm_mhz": 2000.0})
    # 12 MB in 2 ms = 6 GB/s of 6000 GB/s
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(6.0)
    assert r["frac"] == pytest.approx(0.001)
    assert r["traffic"] is None
    assert r["bytes_per_launch"] == pytest.approx(2e6)
    assert r["launch_ms"] == pytest.approx(2e-3 * 1e3 / 6)


def test_alu_roofline_from_counters(monkeypatch):
    rec = {"levels": [1, 2], "dram_bytes": [1e6, 3e6], "alu_warp_inst": [3e5, 9e5],
           "alu_peak_warp_inst_per_sm_cycle": 2.0, "alu_pct_of_peak": [50.0, 60.0]}
    monkeypatch.setattr(bench, "expand_counters", lambda: rec)
    r = bench.roofline_of(_stats(), {"hbm_gbs": 6000.0}, {"sm_mhz": 2000.0})
    # the captured launches (levels 1 and 2: 300 input states) moved 4 MB and
    # 1.2e6 ALU warp-instructions: per input state 13,333 B and 4000; the
    # step's 600 states over 6 launches give 1.333 MB per launch and 2.4e6
    # ALU warp-instructions in 2 ms = 1.2 G/s against 2 x 152 x 2000 MHz
    assert r["bound"] == "alu"
    assert r["traffic"] == pytest.approx(4e6 / 300 * 600 / 6, rel=1e-3)
    assert r["achieved"] == pytest.approx(1.2, rel=1e-3)
    assert r["peak"] == pytest.approx(2.0 * 152 * 2000e6 / 1e9, rel=1e-3)
    assert r["frac"] == round(1.2 / 608.0, 4)  # (reported to four decimals)
    assert r["hbm"]["traffic_over_algorithmic"] == pytest.approx(r["traffic"] / 2e6, rel=1e-2)
    assert r["alu_frac_ncu_captured"] == [0.5, 0.6]


def test_counter_record_from_ncu_csv(tmp_path, monkeypatch):
    metrics = {"gpu__time_duration.sum": ("nsecond", [1000.0, 2000.0]),
               "dram__bytes_read.sum": ("byte", [10.0, 20.0]),
               "dram__bytes_write.sum": ("byte", [1.0, 2.0]),
               "sm__inst_executed_pipe_alu.sum": ("inst", [5.0, 6.0]),
               "smsp__inst_executed.sum": ("inst", [7.0, 8.0]),
               "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active": ("%", [40.0, 45.0]),
               "sm__inst_executed_pipe_alu.avg.peak_sustained": ("inst/cycle", [2.0, 2.0])}
    lines = ['==PROF== log line that is not CSV',
             '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for launch in range(2):
        for name, (unit, vals) in metrics.items():
            lines.append(f'"{launch}","void graph_expand_kernel<unsigned long long, 4, 0>(...)","{name}","{unit}",'
                         f'"{vals[launch]:,}"')
    csv_path = tmp_path / "counters.csv"
    csv_path.write_text("\n".join(lines) + "\n")
    out = tmp_path / "record.json"
    monkeypatch.setattr(bench, "COUNTERS", str(out))
    rec = bench.write_counter_record(str(csv_path), 19, "ncu ...")
    assert rec["levels"] == [19, 20]
    assert rec["dram_bytes"] == [11.0, 22.0]
    assert rec["alu_warp_inst"] == [5.0, 6.0]
    assert rec["warp_inst"] == [7.0, 8.0]
    assert rec["duration_ns"] == [1000.0, 2000.0]
    assert rec["alu_peak_warp_inst_per_sm_cycle"] == 2.0
    assert rec["source_sha256"] == bench.kernel_source_hash()
    assert json.loads(out.read_text())["levels"] == [19, 20]


def test_committed_counter_record_matches_the_kernel_sources():
    # the record the bench reads belongs to the expand kernel as it is now
    rec = bench.expand_counters()
    assert rec is not None and rec["levels"] == [19, 20, 21]
