"""The reference arm of bench.py (the CPU oracle on a bounded sample): one JSON line with
the contract's keys, run on the host only.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line(native_cpu):
    d = run_bench("--impl", "reference", "--workload", "tiny_plain_prefix400", "--steps", "2",
                  "--warmup", "1")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["n_gpus"] == 1 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "tiny_plain_prefix400"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    e2e = d["e2e"]
    assert (e2e["value"], e2e["unit"]) == (d["value"], d["unit"])
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly(native_cpu):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny_plain_prefix400", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_dram_rate():
    sys.path.insert(0, ROOT)
    import bench

    r = bench.dram_rate(5.0e9, 10.0, 6791.0)   # 5 GB in 10 ms
    assert r["dram_achieved"] == 500.0 and r["dram_frac"] == round(500.0 / 6791.0, 4)
    assert bench.dram_rate(None, 10.0, 6791.0) == {}
    assert bench.dram_rate(5.0e9, 0.0, 6791.0) == {}


def test_reference_arm_batched(native_cpu):
    d = run_bench("--impl", "reference", "--workload", "batched", "--batch-members", "2",
                  "--steps", "2", "--warmup", "0")
    assert d["impl"] == "reference" and d["config"]["workload"] == "batched_2"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
