"""bench.py's contract on the host, no GPU: the reference arm's line for a
workload the oracle does not time, and the cpu_baseline leg (the oracle as it
stands, one spawn process per core) on a short sample of the 120-bus grid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_says_unavailable_and_exits_zero():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "pack256"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and "pack256" in d["unavailable"]


def test_cpu_baseline_leg_on_a_short_sample(oracle):
    sys.path.insert(0, ROOT)
    import bench
    r = bench.cpu_baseline("plain120", 0.5, 1)
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert r["cores"] == (os.cpu_count() or 1)
    assert r["value"] > 0 and "120-bus" in r["sample"]
