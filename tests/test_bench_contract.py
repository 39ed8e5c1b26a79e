"""The bench's JSON line for the reference arm, produced on the host cores
(the FP64 oracle; no GPU): one line with every key the benchmark contract
names, on a tiny R-MAT graph (scale 10, 20 queries) so it runs in seconds.
Also the workload label, which follows the arguments a run was given."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def test_reference_arm_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scale", "10",
           "--queries", "20", "--steps", "3", "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["unit"] == "seeds/s" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "R-MAT scale 10" in d["config"]["workload"] and "20 single-seed queries" in d["config"]["workload"]
    assert d["config"]["n"] == 1 << 10 and d["config"]["m"] > 0


def test_workload_label_follows_arguments():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.workload(bench.parse_args([])) == (
        "TPA preprocessing + 1000 single-seed queries on R-MAT scale 22 (ef 16), c=0.15 S=5 T=10 eps=1e-9")
    a = bench.parse_args(["--scale", "26", "--edge-factor", "28", "--queries", "64"])
    assert "64 single-seed queries on R-MAT scale 26 (ef 28)" in bench.workload(a)


def test_reference_arm_config_matches_ours():
    """Both arms print the same config dict (bench_config), and the reference
    arm names the host it ran on."""
    sys.path.insert(0, ROOT)
    import bench
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scale", "10",
           "--queries", "20", "--steps", "3", "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    args = bench.parse_args(["--scale", "10", "--queries", "20"])
    mine = bench.bench_config(args, d["config"]["n"], d["config"]["m"], d["config"]["m_raw"], 1)
    assert d["config"] == mine
    host = d["cpu_baseline"]["host"]
    assert host["nproc"] >= 1 and isinstance(host["model"], str)


def test_contract_bytes():
    """8m + 20n per SpMV and 8m + 4n + 16nk per k-column SpMM."""
    sys.path.insert(0, ROOT)
    import bench
    n, m = 4_194_304, 65_243_475
    assert bench.s8d_bytes(n, m, 1) == 8 * m + 20 * n
    assert bench.s8d_bytes(n, m, 8) == 8 * m + 4 * n + 16 * n * 8
    assert abs(bench.s8d_bytes(n, m, 8) / 1e9 - 1.0756) < 1e-3
