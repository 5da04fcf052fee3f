"""Host-side logic of bench.py that needs no GPU: the clock record, the
traffic record's source check, the algorithmic work, and the reference arm
(the CPU oracle) printing the contract's JSON line."""
import hashlib
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_summary_median_under_load_and_reasons():
    lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active\n",
        "2055, 2070, 1100.0, Not Active, Not Active, Not Active, Active\n",
        "1980, 2070, 1200.0, Not Active, Not Active, Not Active, Active\n",
        "345, 2070, 95.0, Not Active, Not Active, Not Active, Not Active\n",   # idle sample, not under load
        "garbage line\n",
    ]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == 2055.0            # median of the three loaded samples
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    lines.append("2070, 2070, 1000.0, Active, Not Active, Active, Not Active\n")
    assert bench.summarize_clocks(lines)["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.summarize_clocks(["x\n"]) is None


def test_traffic_record_only_for_the_captured_source(tmp_path):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel\n")
    rec = tmp_path / "traffic.json"
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    rec.write_text(json.dumps({"offset": {"source_sha256_16": h, "bytes_per_launch": 1234}}))
    assert bench.traffic_for(str(src), str(rec)) == 1234
    assert bench.traffic_for(str(src), str(rec), workload="wide_range") is None
    src.write_text("// kernel, changed\n")
    assert bench.traffic_for(str(src), str(rec)) is None
    assert bench.traffic_for(str(src), str(tmp_path / "missing.json")) is None


def test_committed_traffic_records_are_consistent():
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, rec in recs.items():
        assert name in bench.WORKLOADS
        assert rec["bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]


def test_column_block_widths_and_issued_flops():
    assert bench.column_block_widths(500, 10) == [128, 128, 128, 128]
    assert bench.column_block_widths(1024, 16, narrow=True) == [128] * 8 + [32]   # 17 used columns -> 32
    assert bench.column_block_widths(1024, 16, narrow=False) == [128] * 9
    assert not bench.narrow_last_block("fp16x3", 1_000_000, 20)
    assert bench.narrow_last_block("tf32", 1_000_000, 20) and bench.narrow_last_block("fp16x3", 50_000, 5000)
    assert bench.column_block_widths(127, 0) == [128]
    assert bench.split_issued_flops([128, 128, 128, 128], 100_000) == bench.issued_mma_flops(100_000, 500, 10)


def test_algorithmic_flops():
    assert bench.algorithmic_flops(100_000, 500, 10) == 2.0 * 100_000 * 500 * 510


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
