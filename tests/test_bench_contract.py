"""Host checks of the benchmark script (no GPU): the reference arm's JSON
line (the oracle timed on a bounded sample), the workload table against the
configurations it stands for, and the DRAM-traffic record lookup."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("workload", ["stabilized20x25", "condensed300"])
def test_reference_arm_json_line(workload):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                          "--steps", "1", "--warmup", "1", "--cpu-side", "16", "--cpu-budget", "0.3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]


def test_workload_table_matches_the_configurations():
    want = {"stabilized20x25": (0, 1e4, 1), "condensed300": (1, 1e5, 1), "batch64": (0, 1e4, 4),
            "adjoint256": (0, 1e4, 1), "large700": (0, 1e6, 1)}
    assert set(bench.WORKLOADS) == set(want)
    for name, (form, rho, nrhs) in want.items():
        spec = bench.workload_spec(name, None)
        assert (spec["form"], spec["rho"], spec["nrhs"]) == (form, rho, nrhs), name
    assert bench.workload_spec("condensed300", 1e8)["rho"] == 1e8


def test_recorded_traffic_only_for_its_workload_and_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    assert rec
    for kernel, r in rec.items():
        assert bench.recorded_traffic(kernel, "large700") is None or r["workload"] == "large700"
        fresh = hashlib.sha256(open(os.path.join(ROOT, r["source"]), "rb").read()).hexdigest() == r["source_sha256"]
        got = bench.recorded_traffic(kernel, r["workload"])
        assert got == (r["traffic_bytes_per_launch"] if fresh else None), kernel
    assert bench.recorded_traffic("no_such_kernel", "condensed300") is None


def test_tuned_table_default_and_overrides():
    """The committed table is applied by default; 'none' or an explicit
    cut-over setting turns it off (the table would override the setting)."""
    assert bench.parse([]).tuned == bench.TUNED
    assert bench.parse(["--tuned", "none"]).tuned is None
    assert bench.parse(["--subtree-sweeps", "1"]).tuned is None
    assert bench.parse(["--persistent-fronts", "0"]).tuned is None
    assert bench.parse(["--tuned", "x.txt"]).tuned == "x.txt"

