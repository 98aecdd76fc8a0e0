"""Host-side checks of bench.py: the reference arm's JSON line (the oracle, no GPU needed) and
the kernel source hash that ties committed DRAM-traffic figures to the sources they came from."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "records/s" and d["unit"] == "records/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "uniform_1e9_r16"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "records/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_source_hash_ignores_comments_only():
    code = "int f(int x) {\n  return x + 1;  // one more\n}\n/* a block\n comment */\n"
    same = "int f(int x) {\n  return x + 1;\n}\n"
    other = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)


def test_committed_traffic_needs_the_same_workload():
    # a figure is only reported for the workload it was captured on
    assert bench.committed_traffic("scatter", "no_such_workload") is None
