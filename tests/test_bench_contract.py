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


def test_accuracy_leg_against_the_oracle_itself(oracle):
    """The accuracy part of the cpu_baseline leg on the 120-bus grid: fed the
    oracle's own tight solution it reports errors at rounding level, and the
    per-case lists have one entry per case."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_1811_02512_gb300 import gridgen
    case = gridgen.config(0)
    rc, vm, va, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-12, max_iter=30)
    acc = bench.oracle_accuracy("plain120", vm[None], va[None], 1)
    assert acc["cases"] == 1 and acc["oracle_failed"] == 0
    assert acc["max_dV_pu"] <= 1e-12 and acc["max_dtheta_rad"] <= 1e-12
    assert len(acc["per_case_dV_pu"]) == 1 and len(acc["per_case_dtheta_rad"]) == 1
    acc = bench.oracle_accuracy("plain120", vm[None] + 1e-6, va[None], 1)
    assert abs(acc["max_dV_pu"] - 1e-6) < 1e-9
