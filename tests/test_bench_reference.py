"""The benchmark's reference arm (the CPU oracle timed on the host) prints the
contract's JSON line for the phi-product and integrator workloads; no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_reference_arm_phiv_line():
    d = run_reference("--config", "0", "--steps", "2", "--cpu-budget", "2")
    assert d["impl"] == "reference" and d["unit"] == "phiv/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_reference_arm_integrator_line():
    d = run_reference("--config", "5", "--size", "32", "--steps", "1", "--cpu-budget", "2")
    assert d["impl"] == "reference" and d["unit"] == "integrator steps/s" and d["value"] > 0
    assert d["config"]["method"] == "epi4"
