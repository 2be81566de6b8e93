"""The benchmark's reference arm (the oracle timed on the host cores) keeps the JSON-line
contract on a CPU-only machine: one line with the metric, unit, direction, the `impl` tag, a
`cpu_baseline` of kind "oracle" and an `e2e` object without host-device copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-cells", "64"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "cells/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"].startswith("chem-step cells/s")
    assert d["config"]["workload"] == "di_c_30sp_1m" and d["config"]["cells_per_step"] == 64
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["unit"] == "cells/s"
    assert d["e2e"] == {"value": d["value"], "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
