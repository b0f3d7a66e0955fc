"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints one JSON line in the benchmark's format."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

COMMON = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
          "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", *extra], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,unit,higher", [("stis", "iterations/s", True), ("wide", "iterations/s", True),
                                                   ("aux", "ms", False)])
def test_reference_arm_prints_one_json_line(workload, unit, higher):
    d = _run("--workload", workload)
    for k in COMMON:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == unit and d["higher_is_better"] is higher
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
