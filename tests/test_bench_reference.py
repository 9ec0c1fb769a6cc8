"""bench.py's reference arm (the FP64 oracle timed on the host) runs on the
CPU: its JSON line follows the bench contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--workload", "single_gauss_16k"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == "atoms/s" and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "single_gauss_16k"
    # the same work and config keys as the GPU arm: the decomposition to the
    # workload's own stop (K = 500 here), analysis named
    assert line["atoms_per_step"] == 500
    assert line["config"]["analysis"] == "fp32" and line["config"]["parallelism"] == "single"
    assert line["cpu_baseline"]["host"]["nproc"] >= 1
