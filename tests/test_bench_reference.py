"""The benchmark's reference arm on CPU: the oracle, timed on a bounded sample of the
headline workload, prints one JSON line with the fields the benchmark contract names
(its own metric, unit and direction, the CPU baseline it describes, and an end-to-end
entry without host-device copies)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["unit"] == "edges/s" and rec["higher_is_better"] is True
    assert rec["value"] > 0 and rec["steps"] == 1 and rec["n_gpus"] == 1
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["cpu_baseline"]["value"] == rec["value"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert rec["config"]["workload"] == "girg_d2_n1e6_T0.5_deg10"


def test_cpu_baseline_one_core_and_all_cores():
    """The CPU baseline: the oracle on one core, and independent samples on every host
    core in spawned processes (the batch's edges over its wall time)."""
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.cpu_baseline(bench.WORKLOAD)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    ac = cb["all_cores"]
    assert ac["cores"] == bench.host_cores() and ac["value"] > 0 and ac["unit"] == "edges/s"
